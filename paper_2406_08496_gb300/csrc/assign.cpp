// Host side of the traffic-assignment loop around the simulator: the
// method of successive averages (MSA) with time-dependent shortest paths.
//
// The paper's title is traffic *assignment* and propagation; its simulator
// propagates trips along routes computed beforehand (Sec. 3.1) and it names
// dynamic rerouting as future work (Sec. 5, Conclusion).  This engine closes
// the loop: link travel times per 15-minute entry bin come from a simulation
// (or from the surrogate), time-dependent shortest paths are computed under
// them (label-setting Dijkstra on earliest arrival, FIFO bin lookup of the
// link time at the entry time), and a fraction of trips is moved onto the
// new paths.  The relative gap is the textbook one,
//   RG = sum_trips (t_experienced - t_shortest) / sum_trips t_shortest.
// Shortest-path trees are shared by trips with the same origin and
// departure period; origins are distributed over POSIX threads and each
// tree is deterministic, so results do not depend on the thread count.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <numeric>
#include <queue>
#include <random>
#include <string>
#include <thread>
#include <vector>

#include "../../include/lpsim_assign.h"
#include "assign_internal.h"
#include "host_par.h"

int lpsim_fail(int code, const std::string &msg);

namespace {
int fail(int code, const std::string &m) { return lpsim_fail(code, m); }
using namespace lpsim_assign_detail;
}  // namespace

namespace {

using lpsim::kPiece;
using lpsim::parallel_pieces;

// Time-dependent Dijkstra from s departing at t0.  want[v] == stamp marks the
// n_want nodes the caller needs; the search stops once all of them are
// settled (their arrival times and predecessor chains are final then: a
// settled node's predecessor was settled before it).
using HeapItem = std::pair<uint64_t, uint32_t>;

// Min-heap of (arrival time, node) pairs with four children per node
// (shallower than a binary heap: fewer levels to sift through per push and
// pop), ordered like the pairs themselves; its storage is the caller's.
struct Heap4 {
    std::vector<HeapItem> &h;
    bool empty() const { return h.empty(); }
    void push(const HeapItem &x) {
        size_t i = h.size();
        h.push_back(x);
        while (i > 0) {
            const size_t p = (i - 1) >> 2;
            if (!(x < h[p])) break;
            h[i] = h[p];
            i = p;
        }
        h[i] = x;
    }
    HeapItem pop() {
        const HeapItem top = h[0];
        const HeapItem x = h.back();
        h.pop_back();
        const size_t n = h.size();
        if (n == 0) return top;
        size_t i = 0;
        for (;;) {
            const size_t c0 = 4 * i + 1;
            if (c0 >= n) break;
            size_t m = c0;
            const size_t c1 = std::min(c0 + 4, n);
            for (size_t c = c0 + 1; c < c1; c++)
                if (h[c] < h[m]) m = c;
            if (!(h[m] < x)) break;
            h[i] = h[m];
            i = m;
        }
        h[i] = x;
        return top;
    }
};

constexpr uint64_t kUnreached = ~0ull;

void td_dijkstra(const TD &td, uint32_t s, uint64_t t0, std::vector<uint64_t> &arr, std::vector<uint32_t> &pred,
                 std::vector<uint8_t> &done, const std::vector<uint32_t> &want, uint32_t stamp, uint32_t n_want,
                 std::vector<HeapItem> &heap) {
    const lpsim_assign *a = td.a;
    std::fill(arr.begin(), arr.end(), kUnreached);
    std::fill(pred.begin(), pred.end(), UINT32_MAX);
    std::fill(done.begin(), done.end(), 0);
    // a min-heap on the caller's storage (kept between searches)
    heap.clear();
    Heap4 pq{heap};
    arr[s] = t0;
    pq.push({t0, s});
    while (!pq.empty()) {
        const auto [t, u] = pq.pop();
        if (done[u]) continue;
        done[u] = 1;
        if (want[u] == stamp && --n_want == 0) break;
        for (uint32_t j = a->out_off[u]; j < a->out_off[u + 1]; j++) {
            const uint32_t e = a->out_edge[j], v = a->dst[e];
            if (done[v]) continue;
            const uint64_t nt = td.arrive(e, t);
            if (nt < arr[v] || (nt == arr[v] && e < pred[v])) {
                arr[v] = nt;
                pred[v] = e;
                pq.push({nt, v});
            }
        }
    }
}

}  // namespace

extern "C" {

int lpsim_assign_create(lpsim_assign **out, uint32_t n_nodes, uint32_t n_edges, const uint32_t *src,
                        const uint32_t *dst, const float *len_m, const uint8_t *lanes, const float *vmax,
                        uint64_t n_trips, const uint32_t *orig, const uint32_t *dest, const uint32_t *depart_step,
                        const uint64_t *route_off, const uint32_t *route_edges, float dt, uint64_t seed) {
    if (!out || !src || !dst || !len_m || !lanes || !vmax || !orig || !dest || !depart_step || !route_off ||
        !route_edges)
        return fail(LPSIM_E_INVALID_ARG, "NULL argument");
    if (!(dt > 0.0f)) return fail(LPSIM_E_INVALID_ARG, "dt must be > 0");
    auto *a = new (std::nothrow) lpsim_assign();
    if (!a) return fail(LPSIM_E_OOM, "host allocation failed");
    a->n_nodes = n_nodes;
    a->n_edges = n_edges;
    a->src.assign(src, src + n_edges);
    a->dst.assign(dst, dst + n_edges);
    a->len.assign(len_m, len_m + n_edges);
    a->vmax.assign(vmax, vmax + n_edges);
    a->lanes.assign(lanes, lanes + n_edges);
    a->out_off.assign(n_nodes + 1, 0);
    for (uint32_t e = 0; e < n_edges; e++) {
        if (src[e] >= n_nodes || dst[e] >= n_nodes) {
            delete a;
            return fail(LPSIM_E_INVALID_ARG, "edge endpoint out of range");
        }
        a->out_off[src[e] + 1]++;
    }
    for (uint32_t i = 0; i < n_nodes; i++) a->out_off[i + 1] += a->out_off[i];
    a->out_edge.resize(n_edges);
    std::vector<uint32_t> fill(a->out_off.begin(), a->out_off.end() - 1);
    for (uint32_t e = 0; e < n_edges; e++) a->out_edge[fill[src[e]]++] = e;
    a->n = n_trips;
    a->orig.assign(orig, orig + n_trips);
    a->dest.assign(dest, dest + n_trips);
    a->dep.assign(depart_step, depart_step + n_trips);
    a->route.resize(n_trips);
    a->cand.resize(n_trips);
    a->tsp.assign(n_trips, 0.0f);
    a->excess.assign(n_trips, 0.0f);
    for (uint64_t j = 0; j < n_trips; j++) {
        if (route_off[j + 1] <= route_off[j] || orig[j] >= n_nodes || dest[j] >= n_nodes) {
            delete a;
            return fail(LPSIM_E_INVALID_ARG, "trip " + std::to_string(j) + ": empty route or bad node");
        }
        a->route[j].assign(route_edges + route_off[j], route_edges + route_off[j + 1]);
    }
    a->dt = dt;
    a->seed = seed;
    *out = a;
    return LPSIM_OK;
}

int lpsim_assign_shortest_paths(lpsim_assign *a, const float *tt, uint32_t n_bins, uint32_t bin_steps,
                                uint32_t period_steps, uint32_t n_threads, float *t_sp) {
    if (!a || !tt || n_bins == 0 || bin_steps == 0 || period_steps == 0)
        return fail(LPSIM_E_INVALID_ARG, "bad argument");
    const TD td(a, tt, n_bins, bin_steps);
    // group trips by (origin, departure period)
    std::vector<uint64_t> order, gstart;
    group_trips(a, period_steps, order, gstart);
    const uint64_t ng = gstart.size() - 1;
    std::atomic<uint64_t> next{0};
    std::atomic<int> bad{0};
    auto worker = [&]() {
        std::vector<uint64_t> arr(a->n_nodes);
        std::vector<uint32_t> pred(a->n_nodes);
        std::vector<uint8_t> done(a->n_nodes);
        std::vector<uint32_t> want(a->n_nodes, 0);
        std::vector<HeapItem> heap;
        std::vector<uint32_t> tmp;
        for (;;) {
            const uint64_t g = next.fetch_add(1);
            if (g >= ng) break;
            const uint64_t j0 = order[gstart[g]];
            const uint32_t s = a->orig[j0];
            const uint32_t period = a->dep[j0] / period_steps;
            // tree from the middle of the departure period
            const uint64_t t0 = period_root_ms(a, period, period_steps);
            // the group's destinations, marked with a stamp unique to the group
            const uint32_t stamp = (uint32_t)g + 1u;
            uint32_t n_want = 0;
            for (uint64_t i = gstart[g]; i < gstart[g + 1]; i++) {
                const uint32_t d = a->dest[order[i]];
                if (want[d] != stamp) {
                    want[d] = stamp;
                    n_want++;
                }
            }
            td_dijkstra(td, s, t0, arr, pred, done, want, stamp, n_want, heap);
            for (uint64_t i = gstart[g]; i < gstart[g + 1]; i++) {
                const uint64_t j = order[i];
                const uint32_t d = a->dest[j];
                if (arr[d] == kUnreached || d == s) {
                    bad = 1;
                    continue;
                }
                tmp.clear();
                for (uint32_t v = d; v != s;) {
                    const uint32_t e = pred[v];
                    tmp.push_back(e);
                    v = a->src[e];
                }
                a->cand[j].assign(tmp.rbegin(), tmp.rend());
                // the tree's path, timed from the trip's own departure (the
                // same start as its experienced time)
                const uint64_t tj = to_ms((double)a->dep[j] * a->dt);
                uint64_t tt_j = tj;
                for (uint32_t e : a->cand[j]) tt_j = td.arrive(e, tt_j);
                a->tsp[j] = (float)((double)(tt_j - tj) / 1000.0);
            }
        }
    };
    const uint32_t nt = std::max<uint32_t>(1, std::min<uint32_t>(n_threads ? n_threads : 1, 256));
    std::vector<std::thread> th;
    for (uint32_t i = 0; i < nt; i++) th.emplace_back(worker);
    for (auto &t : th) t.join();
    if (bad) return fail(LPSIM_E_INVALID_ARG, "a destination is unreachable from its origin");
    if (t_sp) std::memcpy(t_sp, a->tsp.data(), a->n * 4);
    return LPSIM_OK;
}

int lpsim_assign_gap(lpsim_assign *a, const uint32_t *depart_actual, const uint32_t *arrive_step, double *rg,
                     uint64_t *n_used) {
    if (!a || !depart_actual || !arrive_step || !rg) return fail(LPSIM_E_INVALID_ARG, "NULL argument");
    const uint64_t np = (a->n + kPiece - 1) / kPiece;
    std::vector<double> pnum(np, 0.0), pden(np, 0.0);
    std::vector<uint64_t> pused(np, 0);
    parallel_pieces(a->n, [&](uint64_t j0, uint64_t j1, uint64_t p) {
        for (uint64_t j = j0; j < j1; j++) {
            a->excess[j] = 0.0f;
            if (arrive_step[j] == 0xFFFFFFFFu || depart_actual[j] == 0xFFFFFFFFu) continue;
            // experienced time: from the planned departure (waiting to enter counts) to arrival
            const double texp = (double)(arrive_step[j] - a->dep[j]) * a->dt;
            pnum[p] += texp - a->tsp[j];
            pden[p] += a->tsp[j];
            a->excess[j] = (float)(texp - a->tsp[j]);
            pused[p]++;
        }
    });
    double num = 0.0, den = 0.0;
    uint64_t used = 0;
    for (uint64_t p = 0; p < np; p++) {
        num += pnum[p];
        den += pden[p];
        used += pused[p];
    }
    *rg = den > 0 ? num / den : 0.0;
    if (n_used) *n_used = used;
    return LPSIM_OK;
}

int lpsim_assign_reroute(lpsim_assign *a, double fraction, uint32_t iteration, uint64_t *n_changed) {
    if (!a || !(fraction >= 0.0 && fraction <= 1.0)) return fail(LPSIM_E_INVALID_ARG, "bad argument");
    std::mt19937_64 gen(a->seed * 1000003ull + iteration);
    std::uniform_real_distribution<double> u(0.0, 1.0);
    uint64_t changed = 0;
    for (uint64_t j = 0; j < a->n; j++) {
        if (u(gen) >= fraction || a->cand[j].empty()) continue;
        if (a->cand[j] != a->route[j]) {
            a->route[j] = a->cand[j];
            changed++;
        }
    }
    if (n_changed) *n_changed = changed;
    return LPSIM_OK;
}

int lpsim_assign_route_excess(lpsim_assign *a, const float *tt, uint32_t n_bins, uint32_t bin_steps) {
    if (!a || !tt || n_bins == 0 || bin_steps == 0) return fail(LPSIM_E_INVALID_ARG, "bad argument");
    const TD td(a, tt, n_bins, bin_steps);
    parallel_pieces(a->n, [&](uint64_t j0, uint64_t j1, uint64_t) {
        for (uint64_t j = j0; j < j1; j++) {
            const uint64_t t0 = to_ms((double)a->dep[j] * a->dt);
            uint64_t t = t0;
            for (uint32_t e : a->route[j]) t = td.arrive(e, t);
            a->excess[j] = (float)((double)(t - t0) / 1000.0 - a->tsp[j]);
        }
    });
    return LPSIM_OK;
}

int lpsim_assign_reroute_worst(lpsim_assign *a, double fraction, double min_rel_excess, uint64_t *n_changed) {
    if (!a || !(fraction >= 0.0 && fraction <= 1.0) || !(min_rel_excess >= 0.0))
        return fail(LPSIM_E_INVALID_ARG, "bad argument");
    auto rel = [&](uint64_t j) { return (double)a->excess[j] / std::max(1.0, (double)a->tsp[j]); };
    // trips whose candidate differs from their route and whose route is worse
    // than it by more than min_rel_excess, by relative excess (largest first,
    // ties to the lower index)
    std::vector<uint64_t> pick;
    for (uint64_t j = 0; j < a->n; j++)
        if (!a->cand[j].empty() && a->excess[j] > 0.0f && rel(j) > min_rel_excess && a->cand[j] != a->route[j])
            pick.push_back(j);
    const uint64_t want = std::min<uint64_t>(pick.size(), (uint64_t)std::llround(fraction * (double)a->n));
    std::partial_sort(pick.begin(), pick.begin() + want, pick.end(), [&](uint64_t x, uint64_t y) {
        const double rx = rel(x), ry = rel(y);
        return rx != ry ? rx > ry : x < y;
    });
    for (uint64_t i = 0; i < want; i++) a->route[pick[i]] = a->cand[pick[i]];
    if (n_changed) *n_changed = want;
    return LPSIM_OK;
}

uint64_t lpsim_assign_route_length(const lpsim_assign *a) {
    if (!a) return 0;
    uint64_t t = 0;
    for (auto &r : a->route) t += r.size();
    return t;
}

int lpsim_assign_get_routes(const lpsim_assign *a, uint64_t *route_off, uint32_t *route_edges, uint64_t capacity) {
    if (!a || !route_off || !route_edges) return fail(LPSIM_E_INVALID_ARG, "NULL argument");
    if (capacity < lpsim_assign_route_length(a)) return fail(LPSIM_E_INVALID_ARG, "route buffer too small");
    uint64_t o = 0;
    for (uint64_t j = 0; j < a->n; j++) {
        route_off[j] = o;
        std::memcpy(route_edges + o, a->route[j].data(), a->route[j].size() * 4);
        o += a->route[j].size();
    }
    route_off[a->n] = o;
    return LPSIM_OK;
}

int lpsim_assign_load(const lpsim_assign *a, const float *tt, uint32_t n_bins, uint32_t bin_steps, uint32_t *inflow) {
    if (!a || !tt || !inflow || n_bins == 0 || bin_steps == 0) return fail(LPSIM_E_INVALID_ARG, "bad argument");
    const TD td(a, tt, n_bins, bin_steps);
    std::memset(inflow, 0, (size_t)a->n_edges * n_bins * 4);
    parallel_pieces(a->n, [&](uint64_t j0, uint64_t j1, uint64_t) {
        for (uint64_t j = j0; j < j1; j++) {
            uint64_t t = to_ms((double)a->dep[j] * a->dt);
            for (uint32_t e : a->route[j]) {
                const uint64_t b = t / td.bin_ms;
                if (b < n_bins) __atomic_fetch_add(&inflow[(size_t)e * n_bins + b], 1u, __ATOMIC_RELAXED);
                t = td.arrive(e, t);
            }
        }
    });
    return LPSIM_OK;
}

}  // extern "C"

namespace {

// the surrogate inputs of cell (e, b) (the layout lpsim_assign_features
// documents); cells[] = cells of every edge, lin(b') = the edge's scaled log
// inflow of bin b'
template <class Lin>
inline void feature_row(const lpsim_assign *a, uint32_t n_bins, const uint32_t *occ, const float *prev_log_ratio,
                        const uint32_t *prev_inflow, const float *cells, uint32_t e, uint32_t b, const Lin &lin,
                        float *x) {
    x[0] = a->len[e] / 1000.0f;
    x[1] = (float)a->lanes[e] / 4.0f;
    x[2] = a->vmax[e] / 30.0f;
    // inflow of this bin and the three before it (log1p(0) = 0 before the first)
    for (int q = 0; q < 4; q++) x[3 + q] = (int64_t)b - q >= 0 ? lin(b - q) : 0.0f;
    x[7] = 10.0f * (float)occ[(size_t)e * n_bins + b] / cells[e];
    // mean occupancy density of the downstream links
    const uint32_t v = a->dst[e];
    float down = 0.0f;
    uint32_t nd = 0;
    for (uint32_t j = a->out_off[v]; j < a->out_off[v + 1]; j++) {
        const uint32_t f = a->out_edge[j];
        down += (float)occ[(size_t)f * n_bins + b] / cells[f];
        nd++;
    }
    x[8] = nd ? 10.0f * down / (float)nd : 0.0f;
    // the reference simulation of the same (edge, bin): its travel-time ratio and inflow
    const size_t i = (size_t)e * n_bins + b;
    x[9] = std::isfinite(prev_log_ratio[i]) ? prev_log_ratio[i] : 0.0f;
    x[10] = std::log1p((float)prev_inflow[i] / (float)a->lanes[e]) / 4.0f;
}

std::vector<float> edge_cells(const lpsim_assign *a) {
    std::vector<float> cells(a->n_edges);
    parallel_pieces(a->n_edges, [&](uint64_t e0, uint64_t e1, uint64_t) {
        for (uint64_t e = e0; e < e1; e++) cells[e] = std::max(1.0f, std::ceil(a->len[e])) * (float)a->lanes[e];
    });
    return cells;
}

}  // namespace

extern "C" {

int lpsim_assign_features(const lpsim_assign *a, uint32_t n_bins, const uint32_t *inflow, const uint32_t *occ,
                          const float *prev_log_ratio, const uint32_t *prev_inflow, float *X, uint32_t n_features) {
    if (!a || !inflow || !occ || !prev_log_ratio || !prev_inflow || !X || n_features != LPSIM_SURROGATE_FEATURES)
        return fail(LPSIM_E_INVALID_ARG, "bad argument");
    // cells of every edge (for the occupancy densities), once
    const std::vector<float> cells = edge_cells(a);
    parallel_pieces(a->n_edges, [&](uint64_t e0, uint64_t e1, uint64_t) {
        std::vector<float> lin(n_bins);  // the edge's scaled log inflow per bin, each computed once
        for (uint32_t e = (uint32_t)e0; e < (uint32_t)e1; e++) {
            for (uint32_t b = 0; b < n_bins; b++)
                lin[b] = std::log1p((float)inflow[(size_t)e * n_bins + b] / (float)a->lanes[e]) / 4.0f;
            for (uint32_t b = 0; b < n_bins; b++)
                feature_row(a, n_bins, occ, prev_log_ratio, prev_inflow, cells.data(), e, b,
                            [&](uint32_t bb) { return lin[bb]; }, X + ((size_t)e * n_bins + b) * n_features);
        }
    });
    return LPSIM_OK;
}

int lpsim_assign_features_rows(const lpsim_assign *a, uint32_t n_bins, const uint32_t *inflow, const uint32_t *occ,
                               const float *prev_log_ratio, const uint32_t *prev_inflow, uint64_t n_rows,
                               const uint64_t *rows, float *X, uint32_t n_features) {
    if (!a || !inflow || !occ || !prev_log_ratio || !prev_inflow || (n_rows && (!rows || !X)) || n_bins == 0 ||
        n_features != LPSIM_SURROGATE_FEATURES)
        return fail(LPSIM_E_INVALID_ARG, "bad argument");
    const uint64_t n_cells = (uint64_t)a->n_edges * n_bins;
    for (uint64_t r = 0; r < n_rows; r++)
        if (rows[r] >= n_cells) return fail(LPSIM_E_INVALID_ARG, "row index beyond n_edges x n_bins");
    const std::vector<float> cells = edge_cells(a);
    parallel_pieces(n_rows, [&](uint64_t r0, uint64_t r1, uint64_t) {
        for (uint64_t r = r0; r < r1; r++) {
            const uint32_t e = (uint32_t)(rows[r] / n_bins), b = (uint32_t)(rows[r] % n_bins);
            // the same scaled log inflow as the all-cells call computes per bin
            feature_row(a, n_bins, occ, prev_log_ratio, prev_inflow, cells.data(), e, b,
                        [&](uint32_t bb) {
                            return std::log1p((float)inflow[(size_t)e * n_bins + bb] / (float)a->lanes[e]) / 4.0f;
                        },
                        X + r * n_features);
        }
    });
    return LPSIM_OK;
}

int lpsim_assign_link_times(const lpsim_assign *a, uint32_t n_bins, const uint32_t *tt_sum, const uint32_t *tt_cnt,
                            float *tt, float *log_ratio) {
    if (!a || !tt_sum || !tt_cnt || !tt || n_bins == 0) return fail(LPSIM_E_INVALID_ARG, "bad argument");
    parallel_pieces(a->n_edges, [&](uint64_t e0, uint64_t e1, uint64_t) {
        for (uint64_t e = e0; e < e1; e++) {
            const float ff = a->len[e] / a->vmax[e];
            for (uint32_t b = 0; b < n_bins; b++) {
                const size_t i = (size_t)e * n_bins + b;
                if (tt_cnt[i]) {
                    const float m = (float)((double)tt_sum[i] / (double)tt_cnt[i] * a->dt);
                    tt[i] = m;
                    if (log_ratio) log_ratio[i] = std::log(std::max(m, 0.5f * ff) / ff);
                } else {
                    tt[i] = ff;
                    if (log_ratio) log_ratio[i] = NAN;
                }
            }
        }
    });
    return LPSIM_OK;
}

int lpsim_assign_times_from_ratio(const lpsim_assign *a, uint32_t n_bins, const float *y, float *tt) {
    if (!a || !y || !tt || n_bins == 0) return fail(LPSIM_E_INVALID_ARG, "bad argument");
    const float ymax = std::log(50.0f);
    parallel_pieces(a->n_edges, [&](uint64_t e0, uint64_t e1, uint64_t) {
        for (uint64_t e = e0; e < e1; e++) {
            const float ff = a->len[e] / a->vmax[e];
            for (uint32_t b = 0; b < n_bins; b++) {
                const size_t i = (size_t)e * n_bins + b;
                tt[i] = ff * std::exp(std::min(std::max(y[i], 0.0f), ymax));
            }
        }
    });
    return LPSIM_OK;
}

void lpsim_assign_destroy(lpsim_assign *a) { delete a; }

}  // extern "C"
