/*
 * lpsim_oracle.h -- plain single-threaded CPU oracle of the per-step vehicle
 * update of "Large Scale Multi-GPU Based Parallel Traffic Simulation for
 * Accelerated Traffic Assignment and Propagation" (Jiang, Sengupta, Demmel,
 * Williams; arXiv 2406.08496).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the reference the GPU library is
 * checked against.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load it; the product path never does.  It shares no code,
 * header or table with the GPU library.
 *
 * What it computes: Algorithm 1 (Vehicle Propagation) with the car-following
 * (IDM), lane-change and gap-acceptance rules of Sec. 3.1 (eqs. Car Following,
 * Lane Change, Gap Acceptance) as a synchronous (Jacobi) update of every
 * vehicle from the state at step k (eq. vehicle_dynamics), on a byte-per-metre
 * lane map (Sec. 3.1, Lane Map: 255 empty, 0..254 speed in m/s).  Where the
 * paper leaves a rule unstated the oracle takes the readings written out in
 * the comments of lpsim_oracle.c (IDM constants, the no-crash clamp, the
 * mandatory-lane-change probability, the critical gaps, the signal plan, the
 * min-id winner of an edge-entry conflict).
 *
 * Status codes: 0 ok, -1 invalid argument, -2 out of memory, -4 wrong call
 * order, -7 invariant violated (two vehicles in one lane-map cell).
 */
#ifndef LPSIM_ORACLE_H
#define LPSIM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_params {
    float dt;                 /* time step, s */
    float a, b, s0, T;        /* IDM: max accel, comfortable decel, standstill gap, headway; delta = 4 */
    float x0;                 /* mandatory lane change horizon, m */
    float g_a, g_b;           /* desired lead / lag gaps, m */
    float alpha_i, alpha_a, alpha_b; /* anticipation times, s */
    float eps_amp;            /* amplitude of the random gap components, m (0 = none) */
    uint64_t seed;            /* seed of the lane-change draws */
    uint32_t bin_steps;       /* steps per link-statistics bin */
    uint32_t n_bins;          /* bins kept per edge */
    float dlc_prob;           /* discretionary lane change: probability per step when it pays (0 = none) */
    float dlc_gain;           /* discretionary lane change: gap gain it needs, m */
} orc_params;

typedef struct orc_sim orc_sim;

/* Vehicle type (Algorithm 1 State: vehicle type V, recorded when the vehicle
 * moves onto an edge; multimodal traffic is the paper's next step, Sec. 5):
 * its own car-following parameters and a top speed.  The free-flow speed of
 * a vehicle on an edge is min(edge limit, vmax) and the IDM uses the type's
 * a, b, s0, T (delta = 4); the no-crash clamp keeps the type's s0. */
typedef struct orc_vehicle_type {
    float a, b, s0, T;  /* IDM: max accel, comfortable decel, standstill gap, headway */
    float vmax;         /* top speed, m/s (in (0, 254]) */
} orc_vehicle_type;

#define ORC_MAX_TYPES 8

/* Network: node i has green_steps[i] steps of green per approach (0 =
 * uncontrolled); edge e goes src[e] -> dst[e], is len_m[e] metres long
 * (ceil'ed to whole cells), has lanes[e] in 1..4 and speed limit vmax[e].
 * approach_rank[e] is the signal phase of edge e at node dst[e] (must be
 * below the node's in-degree); NULL gives every approach its own phase,
 * ranked by edge id among the incoming edges of the node. */
int orc_create(orc_sim **out, uint32_t n_nodes, uint32_t n_edges,
               const uint32_t *src, const uint32_t *dst, const float *len_m,
               const uint8_t *lanes, const float *vmax, const uint32_t *green_steps,
               const uint8_t *approach_rank, const orc_params *p);

/* Trips: depart_step[j] and route j = route_edges[route_off[j] .. route_off[j+1]).
 * Vehicle ids are the ranks of a stable sort by depart_step; out_vid[j]
 * (nullable) receives trip j's id. */
int orc_load_demand(orc_sim *s, uint64_t n_trips, const uint32_t *depart_step,
                    const uint64_t *route_off, const uint32_t *route_edges, uint32_t *out_vid);

/* Vehicle types 0..n_types-1 (n_types <= ORC_MAX_TYPES), before
 * orc_load_demand*; without this call there is one type with the params'
 * a, b, s0, T and vmax 254. */
int orc_set_vehicle_types(orc_sim *s, uint32_t n_types, const orc_vehicle_type *types);

/* orc_load_demand with a type per trip (vtype[j] < the number of types;
 * NULL: every trip type 0). */
int orc_load_demand_typed(orc_sim *s, uint64_t n_trips, const uint32_t *depart_step, const uint64_t *route_off,
                          const uint32_t *route_edges, const uint8_t *vtype, uint32_t *out_vid);

int orc_step(orc_sim *s, uint32_t n_steps);

/* Steps until every trip has arrived or max_steps were taken.  out6 =
 * {steps taken, veh_steps (active vehicle-steps), arrived, active, waiting, k}. */
int orc_run(orc_sim *s, uint32_t max_steps, uint64_t *out6);

/* Per vehicle id: x, v, edge, lane, route index, status (0 waiting,
 * 1 active, 2 arrived). */
int orc_get_state(const orc_sim *s, float *x, float *v, uint32_t *edge, uint8_t *lane,
                  uint32_t *ridx, uint8_t *status);
int orc_get_trips(const orc_sim *s, uint32_t *depart_actual, uint32_t *arrive_step);

/* Lane map at the current step, edges in id order, lanes in order, cells
 * 0..len-1 (no padding). */
uint64_t orc_lane_map_size(const orc_sim *s);
int orc_get_lane_map(const orc_sim *s, uint8_t *out);

/* Per edge: entries, exits, sum of traversal steps (3 x u64 each, interleaved);
 * per (edge, bin): inflow, traversal-step sum and count by entry bin, and
 * vehicles on the edge sampled at the first step of the bin (u32, n_edges x n_bins each). */
int orc_link_stats(const orc_sim *s, uint64_t *per_edge3, uint32_t *bin_inflow, uint32_t *bin_tt_sum,
                   uint32_t *bin_tt_cnt, uint32_t *bin_occ);

/* Totals so far: {k, veh_steps (active vehicle-steps), arrived, active,
 * waiting, accepted lane changes}. */
int orc_counters(const orc_sim *s, uint64_t *out6);

/* The IDM branch of the car-following rule for one vehicle, in the oracle's
 * operation order: speed v, leader byte speed vf, gap s, edge limit v0. */
float orc_idm_speed(const orc_params *p, float v, float vf, float s, float v0);

void orc_destroy(orc_sim *s);

#ifdef __cplusplus
}
#endif
#endif
