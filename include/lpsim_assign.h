/*
 * lpsim_assign.h -- host engine of the traffic-assignment loop around the
 * simulator (method of successive averages with time-dependent shortest
 * paths), and the feature builder of the link-travel-time surrogate.
 *
 * The paper's title names traffic assignment and propagation; its simulator
 * takes the routes as computed beforehand (Sec. 3.1) and it names dynamic
 * rerouting as future work (Sec. 5, Conclusion).  None of these calls has
 * a formula in the paper: the relative gap is the textbook Wardrop gap
 *   RG = sum_trips (t_experienced - t_shortest) / sum_trips t_shortest,
 * t_experienced from planned departure to arrival in the simulation and
 * t_shortest the earliest-arrival path time under the link times of the same
 * simulation.  Link times come per (edge, 15-minute entry bin), rounded to
 * whole milliseconds; entering edge e at time t in bin b arrives at
 *   min(t + c[b][e], min over later bins b' of (start of b' + c[b'][e])),
 * i.e. an entry may be held back to a later bin when that arrives earlier,
 * which makes every link FIFO (a later entry never arrives earlier) and the
 * earliest-arrival searches exact.
 *
 * Conventions as in lpsim.h (status codes, lpsim_last_error(), host
 * pointers, caller-owned buffers).  Everything here runs on the host CPU
 * threads; the simulation and the surrogate run on the GPU.
 */
#ifndef LPSIM_ASSIGN_H
#define LPSIM_ASSIGN_H

#include <stdint.h>

#include "lpsim.h"

#ifdef __cplusplus
extern "C" {
#endif

/* number of surrogate input features per (link, bin): length, lanes, speed
 * limit, inflow in the bin and the 3 bins before it, occupancy of the link
 * and mean occupancy of its downstream links, and -- from the reference
 * simulation the prediction starts from -- the travel-time ratio and the
 * inflow of the same (link, bin) */
#define LPSIM_SURROGATE_FEATURES 11u

typedef struct lpsim_assign lpsim_assign;

/* Network (as in lpsim_network), trips (origin and destination node,
 * departure step) and their initial routes (route_off: n_trips + 1 entries). */
int lpsim_assign_create(lpsim_assign **out, uint32_t n_nodes, uint32_t n_edges, const uint32_t *src,
                        const uint32_t *dst, const float *len_m, const uint8_t *lanes, const float *vmax,
                        uint64_t n_trips, const uint32_t *orig, const uint32_t *dest, const uint32_t *depart_step,
                        const uint64_t *route_off, const uint32_t *route_edges, float dt, uint64_t seed);

/* Time-dependent shortest paths of every trip under link times tt (n_edges x
 * n_bins seconds, bin b covers entry steps [b*bin_steps, (b+1)*bin_steps)).
 * Trips with the same origin and departure period (period_steps) share one
 * earliest-arrival tree rooted at the middle of the period.  Keeps each
 * trip's tree path as its candidate route and, in t_sp (nullable, n_trips
 * entries), that path's travel time (s) when left at the trip's own
 * departure step. */
int lpsim_assign_shortest_paths(lpsim_assign *a, const float *tt, uint32_t n_bins, uint32_t bin_steps,
                                uint32_t period_steps, uint32_t n_threads, float *t_sp);

/* lpsim_assign_shortest_paths with the earliest-arrival trees searched on
 * the GPU (device current at the first call; one warp per tree, thousands of
 * trees at a time, label-correcting rounds on 64-bit (arrival, edge)
 * labels).  Same candidate routes and t_sp, bit for bit, as the host
 * searches: link times are whole milliseconds, so every arrival is an exact
 * sum, and both keep the earliest arrival with ties to the lower entering
 * edge id.  The graph, trip table and search workspaces (32 bytes per node
 * per concurrent tree, up to 40 trees per SM within 48 GiB) stay on the
 * device between calls and are released by lpsim_assign_destroy.  Errors as the host call, plus
 * LPSIM_E_CUDA, LPSIM_E_OOM and LPSIM_E_STATE (another device current). */
int lpsim_assign_shortest_paths_gpu(lpsim_assign *a, const float *tt, uint32_t n_bins, uint32_t bin_steps,
                                    uint32_t period_steps, float *t_sp);

/* Relative gap of the last shortest paths against a simulation's trip
 * outcome (per trip, in the caller's trip order): trips that have not
 * arrived are left out; *n_used counts the others. */
int lpsim_assign_gap(lpsim_assign *a, const uint32_t *depart_actual, const uint32_t *arrive_step, double *rg,
                     uint64_t *n_used);

/* Method of successive averages: each trip moves to its candidate route with
 * probability `fraction` (seeded by the engine seed and `iteration`). */
int lpsim_assign_reroute(lpsim_assign *a, double fraction, uint32_t iteration, uint64_t *n_changed);

/* Per-trip excess of the current route over the shortest path of the last
 * lpsim_assign_shortest_paths call, in seconds, predicted under link times
 * tt (edge-major, n_bins bins of bin_steps steps): the route is traversed from
 * the planned departure with each link's time looked up at its entry time.
 * lpsim_assign_gap sets the same per-trip excess from a simulation's
 * experienced times instead (0 for trips that did not arrive). */
int lpsim_assign_route_excess(lpsim_assign *a, const float *tt, uint32_t n_bins, uint32_t bin_steps);

/* Method of successive averages, worst first: up to round(fraction * n_trips)
 * trips with the largest relative excess (excess / shortest time, the
 * shortest time counted as at least 1 s) move to their candidate route; only
 * trips whose candidate differs and whose relative excess is above
 * min_rel_excess (an indifference band, >= 0) are eligible; ties go to the
 * lower trip index.  *n_changed = trips moved. */
int lpsim_assign_reroute_worst(lpsim_assign *a, double fraction, double min_rel_excess, uint64_t *n_changed);

/* Current routes (route_off: n_trips + 1 entries; route_edges: capacity
 * entries, at least lpsim_assign_route_length()). */
uint64_t lpsim_assign_route_length(const lpsim_assign *a);
int lpsim_assign_get_routes(const lpsim_assign *a, uint64_t *route_off, uint32_t *route_edges, uint64_t capacity);

/* Inflow per (edge, bin) of the current routes propagated with link times tt
 * (departure at the planned step, each link entered at the running time). */
int lpsim_assign_load(const lpsim_assign *a, const float *tt, uint32_t n_bins, uint32_t bin_steps, uint32_t *inflow);

/* lpsim_assign_load with the walk on the GPU (one thread per trip, the
 * routes uploaded for the call): the same counts.  The device state is the
 * one lpsim_assign_shortest_paths_gpu sets up.  Errors as that call. */
int lpsim_assign_load_gpu(const lpsim_assign *a, const float *tt, uint32_t n_bins, uint32_t bin_steps,
                          uint32_t *inflow);

/* Surrogate inputs per (edge, bin), edge-major, LPSIM_SURROGATE_FEATURES
 * floats each, from the inflow counts of the assignment to score, occupancy
 * samples, and the reference simulation's log travel-time ratio (NaN where
 * unmeasured) and inflow (all n_edges x n_bins). */
int lpsim_assign_features(const lpsim_assign *a, uint32_t n_bins, const uint32_t *inflow, const uint32_t *occ,
                          const float *prev_log_ratio, const uint32_t *prev_inflow, float *X, uint32_t n_features);

/* lpsim_assign_features for the listed cells only: row r of X (n_rows x
 * LPSIM_SURROGATE_FEATURES) holds the inputs of cell rows[r] = edge * n_bins
 * + bin, equal bit for bit to that cell's row of the all-cells call (the
 * arrays are the same full n_edges x n_bins inputs).  A cell index beyond
 * n_edges x n_bins is LPSIM_E_INVALID_ARG. */
int lpsim_assign_features_rows(const lpsim_assign *a, uint32_t n_bins, const uint32_t *inflow, const uint32_t *occ,
                               const float *prev_log_ratio, const uint32_t *prev_inflow, uint64_t n_rows,
                               const uint64_t *rows, float *X, uint32_t n_features);

/* Link times (s) per (edge, bin) from a simulation's binned traversal sums
 * and counts; bins without a traversal take the free-flow time len / vmax.
 * log_ratio (nullable) receives log(measured / free-flow) where measured
 * (NaN elsewhere): the surrogate's training target. */
int lpsim_assign_link_times(const lpsim_assign *a, uint32_t n_bins, const uint32_t *tt_sum, const uint32_t *tt_cnt,
                            float *tt, float *log_ratio);

/* Link times from surrogate outputs y = log(t / free-flow), clamped to
 * [free-flow, 50 x free-flow]. */
int lpsim_assign_times_from_ratio(const lpsim_assign *a, uint32_t n_bins, const float *y, float *tt);

void lpsim_assign_destroy(lpsim_assign *a);

#ifdef __cplusplus
}
#endif
#endif
