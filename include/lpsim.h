/*
 * lpsim.h -- C ABI of the GB300 (sm_103a) per-step vehicle update of
 * "Large Scale Multi-GPU Based Parallel Traffic Simulation for Accelerated
 * Traffic Assignment and Propagation" (Jiang, Sengupta, Demmel, Williams;
 * arXiv 2406.08496).
 *
 * What the library computes.  One simulation step moves every vehicle on the
 * network from its state at step k to step k+1 using only step-k state
 * (eq. vehicle_dynamics, Sec. 3.1), following Algorithm 1 (Vehicle
 * Propagation): departure when the first cell of the first edge is free,
 * leader search within d_front = 2 dt v on a byte-per-metre lane map
 * (Sec. 3.1, Lane Map: 255 = empty, 0..254 = speed of the occupying vehicle),
 * IDM car following (eq. Car Following) or the free-flow speed, signal
 * control at the stop line, mandatory lane change (eq. Lane Change) with gap
 * acceptance (eq. Gap Acceptance), and entry to the next edge of the
 * precomputed route when its first cell is free, one vehicle per cell
 * (Sec. 3.1 Remark; Sec. 3.2).  Rules the paper names without a formula use
 * the readings documented with the library: IDM with delta = 4; no-crash
 * clamp at the standstill gap s0; lane-change probability 1 - x_rem/x0;
 * critical gaps g + max(0, alpha_i v - alpha_a v_a) + eps; fixed-time
 * signals (approach of phase j green iff (k / G) mod n_phases == j); several
 * vehicles asking for one (edge, lane) entry: the lowest vehicle id wins.
 * All vehicle state is IEEE binary32 and the results do not depend on
 * launch configuration, sort period or processing order.
 *
 * Conventions.
 *  - Every function returns an int status: LPSIM_OK (0) or a negative
 *    LPSIM_E_* code; lpsim_last_error() gives a message for the calling
 *    thread's last failure.  No C++ exception crosses this boundary.
 *  - Every pointer argument that is an input is a HOST pointer to
 *    caller-owned memory, read during the call and copied; nothing is
 *    retained.  Every output is written into a caller-owned HOST buffer
 *    whose size the caller states; a buffer that is too small gives
 *    LPSIM_E_INVALID_ARG.
 *  - Device memory is owned by the context and released by lpsim_destroy.
 *    It comes from cudaMalloc unless lpsim_set_allocator installed a
 *    callback pair (the Python binding routes it to PyTorch's caching
 *    allocator).
 *  - A context runs on the CUDA stream given to lpsim_load_network on the
 *    device current at that call; NULL makes the library create its own
 *    non-blocking stream (steps are captured into CUDA graphs, which the
 *    legacy default stream cannot do).  Calls on one context must not
 *    overlap.
 */
#ifndef LPSIM_H
#define LPSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LPSIM_OK 0
#define LPSIM_E_INVALID_ARG (-1) /* bad argument or input data (message says which) */
#define LPSIM_E_OOM (-2)         /* device or host allocation failed */
#define LPSIM_E_CUDA (-3)        /* a CUDA runtime call failed */
#define LPSIM_E_STATE (-4)       /* call out of order (e.g. stepping before lpsim_load_demand) */
#define LPSIM_E_TIMEOUT (-5)     /* a bounded device wait gave up */
#define LPSIM_E_GRIDLOCK (-6)    /* vehicles active but none moved for the stated number of steps */
#define LPSIM_E_INVARIANT (-7)   /* device check: a lane-map cell written twice in one step */

#define LPSIM_F_NO_SORT 1u
#define LPSIM_F_CHECK_CELLS 2u
#define LPSIM_F_NO_LIGHT 4u
#define LPSIM_F_SHARED_MAPS 8u

typedef struct lpsim_ctx lpsim_ctx;

/* Model and run parameters.  Model fields mirror the symbols of Table 3. */
typedef struct lpsim_params {
    float dt;          /* time step Delta t, s (> 0) */
    float a;           /* IDM acceleration potential, m/s^2 (> 0) */
    float b;           /* IDM comfortable deceleration, m/s^2 (> 0) */
    float s0;          /* standstill spacing, m (>= 0) */
    float T;           /* desired time headway, s */
    float x0;          /* distance to the edge end below which a mandatory lane change may start, m (> 0) */
    float g_a, g_b;    /* desired lead / lag gaps, m */
    float alpha_i, alpha_a, alpha_b; /* anticipation times of the changer, lead and lag vehicle, s */
    float eps_amp;     /* random gap components eps ~ U(-eps_amp, eps_amp), m; 0 = none */
    uint64_t seed;     /* seed of the lane-change draws (SplitMix64 of seed, vehicle id, step) */
    uint32_t bin_steps;   /* steps per link-statistics bin (0 = no binned statistics) */
    uint32_t n_bins;      /* bins kept per edge */
    uint32_t sort_period; /* steps between re-sorts of the active vehicles by lane-map cell (0 = 256, at most 256) */
    uint32_t block_size;  /* threads per block of the step kernels: 128, 256, 512 or 0 (= 256) */
    uint32_t blocks_per_sm; /* resident 256-thread blocks per SM the step grids are sized for (0 = 4) */
    uint32_t chunk_steps; /* steps captured in one CUDA graph launch (0 = 1536); rounded up to a multiple
                             of 2 sort periods and of 3 */
    uint32_t gridlock_steps; /* lpsim_run fails with LPSIM_E_GRIDLOCK after this many steps with active
                                vehicles and no departure, crossing or arrival (0 = never) */
    uint32_t flags;       /* LPSIM_F_NO_SORT: compact without sorting; LPSIM_F_CHECK_CELLS: check that
                             every lane-map write lands on an empty cell (LPSIM_E_INVARIANT otherwise;
                             costs a load per write); LPSIM_F_NO_LIGHT: never run a chunk in the
                             single-block light-load kernel (results are the same either way);
                             LPSIM_F_SHARED_MAPS: the light-load kernel copies the five lane maps
                             into its shared memory for each chunk when they fit (at most 200 KB:
                             networks of up to ~40k lane-metres; results are the same either way;
                             measured 2% slower on a 4x4 grid, whose maps stay in L2 anyway);
                             other bits must be 0 */
    uint32_t light_trips; /* a chunk runs in the single-block light-load kernel when at most this many
                             trips can be on the network or waiting during it (0 = 1536); a speed
                             setting only, results are the same for every value */
    float dlc_prob;       /* discretionary lane change (an extension; the paper defines only the
                             mandatory change): per-step probability, in [0, 1], that a vehicle
                             outside the mandatory zone, held below its free speed by a slower
                             leader, intends one lane up (odd steps) or down (even steps); 0 = off */
    float dlc_gain;       /* the lead gap in that lane must be absent or longer than the own lane's
                             by at least this many metres (>= 0) */
} lpsim_params;

/* Road network.  Edge e runs edge_src[e] -> edge_dst[e], is edge_len_m[e]
 * metres long (stored as max(1, ceil(len)) one-metre cells per lane, at most
 * 65535), has edge_lanes[e] in 1..4 lanes and speed limit edge_vmax[e] in
 * (0, 254] m/s.  node_green_steps[i] is the green time per phase at node i in
 * steps (0 = uncontrolled).  edge_approach_rank (nullable) is the signal
 * phase of edge e at its downstream node, below that node's in-degree; NULL
 * gives each incoming edge its own phase ranked by edge id.  At most 255
 * incoming and 255 outgoing edges per node. */
typedef struct lpsim_network {
    uint32_t n_nodes, n_edges;
    const uint32_t *edge_src, *edge_dst;
    const float *edge_len_m;
    const uint8_t *edge_lanes;
    const float *edge_vmax;
    const uint32_t *node_green_steps;
    const uint8_t *edge_approach_rank;
} lpsim_network;

typedef struct lpsim_run_result {
    uint64_t steps;     /* steps taken by this call */
    uint64_t veh_steps; /* sum over those steps of the vehicles on the network (active vehicle-steps) */
    uint64_t arrived;   /* trips arrived so far */
    uint64_t active;    /* vehicles on the network now */
    uint64_t waiting;   /* trips not yet departed */
    uint64_t k;         /* current step */
    double wall_ms;     /* host wall time of the call */
} lpsim_run_result;

typedef struct lpsim_link_stat {
    uint64_t entries;  /* vehicles that entered the edge (departures included) */
    uint64_t exits;    /* vehicles that left it (arrivals included) */
    uint64_t tt_steps; /* sum over exits of the steps spent on the edge */
} lpsim_link_stat;

typedef struct lpsim_counters {
    uint64_t k, veh_steps, arrived, active, waiting, lane_changes;
    uint64_t slots;       /* vehicle slots in use (active plus not yet compacted) */
    uint64_t launches;    /* kernel launches issued by this context */
    uint64_t light_chunks; /* chunks run in the single-block light-load kernel */
} lpsim_counters;

/* Message of the calling thread's last failure ("" if none). */
const char *lpsim_last_error(void);

/* Library version string. */
const char *lpsim_version(void);

/* Route this process's device allocations of contexts created afterwards
 * through alloc(size, user) / release(ptr, user); alloc must return memory
 * usable on the current device and aligned to 256 bytes, or NULL.  Both NULL
 * restores cudaMalloc / cudaFree. */
int lpsim_set_allocator(void *(*alloc)(size_t size, void *user), void (*release)(void *ptr, void *user),
                        void *user);

/* Create a context and upload the network (Sec. 3.1, Network Data
 * Information: per edge the lanes, its place in the lane map, upstream and
 * downstream intersection).  stream: a cudaStream_t other than the legacy
 * default stream, or NULL (the library then creates its own stream). */
int lpsim_load_network(lpsim_ctx **out, const lpsim_network *net, const lpsim_params *p, void *stream);

/* Upload the routed trips (Sec. 3.1, Vehicle Data Information: route and
 * first edge "after the routing").  Trip j departs no earlier than step
 * depart_step[j] and follows route_edges[route_off[j] .. route_off[j+1]), a
 * non-empty sequence of edges where each edge starts at the node the previous
 * one ends at.  n_trips may be 0 (an empty demand: steps move nothing and
 * lpsim_run returns at once); depart_step and route_edges may then be NULL.
 * route_off has n_trips + 1 entries starting at 0; the total
 * route length must stay below 2^32.  Vehicle ids are the ranks of a stable
 * sort of the trips by depart_step (the paper sorts by departure time,
 * Sec. 4, Table 6); out_vehicle_id (nullable, n_trips entries) receives trip
 * j's id.  Resets the step counter to 0.  Once per context.  Errors:
 * LPSIM_E_INVALID_ARG when route_off is not increasing from 0 (an empty
 * route), an edge id is out of range or consecutive route edges do not
 * meet; the message names the lowest failing trip, offset errors before edge
 * errors (the checks run on the host's threads); LPSIM_E_STATE on a second
 * call.  The routes are reordered on the host in a staging buffer of 4 bytes
 * per route entry that the process keeps for later loads (one load uses it at
 * a time; it grows to the largest demand loaded and is released at exit). */
int lpsim_load_demand(lpsim_ctx *ctx, uint64_t n_trips, const uint32_t *depart_step, const uint64_t *route_off,
                      const uint32_t *route_edges, uint32_t *out_vehicle_id);

/* Vehicle types (Algorithm 1 State: the vehicle type V, recorded whenever a
 * vehicle moves onto an edge; multimodal traffic is the paper's next step,
 * Sec. 5).  A type carries its own car-following parameters (eq. Car
 * Following: IDM with delta = 4) and a top speed: a vehicle's free-flow
 * speed on an edge (Algorithm 1: v <- v_free) is min(edge limit, vmax), the
 * IDM and the no-crash clamp use the type's a, b, s0, T.  Lane change and
 * gap acceptance do not depend on the type. */
#define LPSIM_MAX_VEHICLE_TYPES 8u
typedef struct lpsim_vehicle_type {
    float a;     /* IDM acceleration potential, m/s^2 (> 0) */
    float b;     /* IDM comfortable deceleration, m/s^2 (> 0) */
    float s0;    /* standstill spacing, m (>= 0) */
    float T;     /* desired time headway, s */
    float vmax;  /* top speed, m/s, in (0, 254] */
} lpsim_vehicle_type;

/* Types 0..n_types-1 (1 <= n_types <= LPSIM_MAX_VEHICLE_TYPES), before
 * lpsim_load_demand_typed.  Without this call every vehicle has the
 * lpsim_params a, b, s0, T and no top speed of its own.  Errors:
 * LPSIM_E_INVALID_ARG on a count or value out of range; LPSIM_E_STATE once
 * trips are loaded. */
int lpsim_set_vehicle_types(lpsim_ctx *ctx, uint32_t n_types, const lpsim_vehicle_type *types);

/* lpsim_load_demand with a vehicle type per trip: vtype[j] (n_trips entries,
 * each below the number of types set; NULL = every trip type 0).  Errors as
 * lpsim_load_demand, plus LPSIM_E_INVALID_ARG on a type out of range. */
int lpsim_load_demand_typed(lpsim_ctx *ctx, uint64_t n_trips, const uint32_t *depart_step, const uint64_t *route_off,
                            const uint32_t *route_edges, const uint8_t *vtype, uint32_t *out_vehicle_id);

/* Advance n_steps steps of Algorithm 1 (Vehicle Propagation, Sec. 3.1-3.2):
 * each step moves every vehicle from its step-k state to step k+1 using only
 * step-k state (eq. vehicle_dynamics, Sec. 3.1) -- departure when the first
 * cell of the first edge is free, leader search within d_front, IDM car
 * following (eq. Car Following) or the free-flow speed, signal control at the
 * stop line, lane change (eq. Lane Change) with gap acceptance (eq. Gap
 * Acceptance), entry to the next route edge one vehicle at a time (Sec. 3.2).
 * Returns after the steps have completed on the device and the device status
 * word was read.  n_steps 0 only reads the status word.  Errors:
 * LPSIM_E_STATE before lpsim_load_demand; LPSIM_E_INVARIANT when the
 * LPSIM_F_CHECK_CELLS check found a lane-map cell written twice or the slot
 * capacity overflowed; LPSIM_E_CUDA when a launch or copy failed (the context
 * is then unusable: destroy it).  A failed call may have taken some of the
 * steps; lpsim_get_counters tells how many. */
int lpsim_step(lpsim_ctx *ctx, uint32_t n_steps);

/* Step (Algorithm 1, as lpsim_step) until every trip has arrived or
 * max_steps steps were taken -- the whole-run simulation whose wall time the
 * paper reports (Sec. 4).  out (nullable) receives the totals of this call:
 * steps taken, vehicle-steps (sum over those steps of the vehicles on the
 * network), trips arrived / active / waiting, the current step and the host
 * wall time.  Errors as lpsim_step, plus LPSIM_E_GRIDLOCK when
 * params.gridlock_steps is non-zero and that many steps passed with vehicles
 * on the network and no departure, crossing or arrival (a host-side check of
 * the device counters after each graph chunk; no kernel waits on it). */
int lpsim_run(lpsim_ctx *ctx, uint32_t max_steps, lpsim_run_result *out);

/* Back to step 0 with the same network and trips (the state before the
 * first step of Algorithm 1: every trip waiting for t_depart, empty lane
 * maps), statistics cleared.  No host-device transfer of inputs.  Errors:
 * LPSIM_E_CUDA. */
int lpsim_reset(lpsim_ctx *ctx);

/* Link statistics, from the step each vehicle entered its current edge
 * (t_start of Algorithm 1, recorded "on a new edge") and the step it left:
 * out (nullable) receives n_edges records {entries, exits, summed steps on the
 * edge}.  The signature is wider than a per-edge query alone: the four binned
 * arrays (each nullable, n_edges * n_bins u32, edge-major; bins of
 * params.bin_steps steps) feed the assignment loop and its travel-time
 * surrogate -- per (edge, bin): inflow counted at entry step k+1 in bin
 * (k+1)/bin_steps; steps spent and exit count of the vehicles that entered in
 * that bin; the vehicles on the edge at the first step of the bin.  Errors:
 * LPSIM_E_INVALID_ARG when n_edges or (with a binned array) n_bins differ from
 * the context's; LPSIM_E_OOM when the device scratch of the binned transpose
 * cannot be allocated; LPSIM_E_CUDA. */
int lpsim_link_stats(lpsim_ctx *ctx, lpsim_link_stat *out, uint64_t n_edges, uint32_t *bin_inflow,
                     uint32_t *bin_tt_sum, uint32_t *bin_tt_cnt, uint32_t *bin_occ, uint32_t n_bins);

/* Per-trip outputs of the simulation (Algorithm 1 State: t_depart; the
 * trip's travel time is what the paper's assignment use rests on, Sec. 1):
 * per vehicle id (n entries each, n = trips loaded) the step at which it
 * entered the network (0xFFFFFFFF if not yet) and the step at which it
 * arrived (0xFFFFFFFF if not yet).  Either pointer may be NULL.  Errors:
 * LPSIM_E_STATE before lpsim_load_demand; LPSIM_E_INVALID_ARG when n differs
 * from the trips loaded; LPSIM_E_CUDA. */
int lpsim_get_trips(lpsim_ctx *ctx, uint64_t n, uint32_t *depart_actual, uint32_t *arrive_step);

/* Vehicle state of Algorithm 1 (Output: position P and speed v) and of the
 * vehicle record of Sec. 3.1 (Vehicle Data Information: current edge,
 * position on it, place in the route): per vehicle id (n entries each, n =
 * trips loaded) position on the edge (m), speed (m/s), edge, lane, index in
 * its route and status (0 waiting, 1 active, 2 arrived); non-active vehicles
 * read x = v = 0, edge 0xFFFFFFFF, lane 0, index 0.  Any pointer may be NULL.
 * Takes n * 17 bytes of device scratch for the call (from cudaMalloc or the
 * allocator callback) and gives it back before returning, on every path.
 * Errors: LPSIM_E_STATE before lpsim_load_demand; LPSIM_E_INVALID_ARG when n
 * differs from the trips loaded; LPSIM_E_OOM; LPSIM_E_CUDA. */
int lpsim_get_state(lpsim_ctx *ctx, uint64_t n, float *x, float *v, uint32_t *edge, uint8_t *lane,
                    uint32_t *route_idx, uint8_t *status);

/* Lane map at the current step (Sec. 3.1, Lane Map: one byte per metre of
 * lane, 255 = empty, 0..254 = speed of the occupying vehicle; lanes of an
 * edge one after the other) in canonical layout: edges in id order, lanes in
 * order, cells 0..len-1, no padding; size = lpsim_lane_map_size() bytes.
 * Errors: LPSIM_E_INVALID_ARG on a NULL pointer or a wrong size. */
uint64_t lpsim_lane_map_size(const lpsim_ctx *ctx);
int lpsim_get_lane_map(lpsim_ctx *ctx, uint8_t *out, uint64_t size);

/* Run counters (no paper counterpart: the quantities the benchmarks report,
 * vehicle-steps above all).  Reads the device status word; errors as
 * lpsim_step. */
int lpsim_get_counters(lpsim_ctx *ctx, lpsim_counters *out);

/* ---- batched scenarios ------------------------------------------------
 * Many independent scenarios (networks with their own trips and lane-change
 * seed) simulated as one: the networks are laid side by side (node, edge and
 * lane-map ids of scenario s follow those of scenario s-1), so one launch of
 * each step kernel advances every scenario.  Vehicles of different scenarios
 * never share an edge, and each vehicle draws its lane-change numbers from
 * its scenario's seed and its id within the scenario, so every scenario's
 * results are identical to simulating it alone.  Query results (link
 * statistics, lane map, per-vehicle arrays) cover the whole batch in
 * scenario order; lpsim_batch_offsets gives where each scenario starts. */
int lpsim_load_network_batch(lpsim_ctx **out, uint32_t n_scen, const lpsim_network *nets, const lpsim_params *p,
                             void *stream);
/* Trips of scenario s: n_trips[s] trips with the arrays of lpsim_load_demand
 * in scenario-local edge ids.  seeds (nullable): lane-change seed per
 * scenario (default p->seed).  out_vehicle_id (nullable): batch vehicle id
 * of every trip, scenarios one after the other. */
int lpsim_load_demand_batch(lpsim_ctx *ctx, uint32_t n_scen, const uint64_t *n_trips,
                            const uint32_t *const *depart_step, const uint64_t *const *route_off,
                            const uint32_t *const *route_edges, const uint64_t *seeds, uint32_t *out_vehicle_id);
/* Prefix offsets (n_scen + 1 entries each, nullable) of nodes, edges,
 * canonical lane-map cells and trips per scenario. */
int lpsim_batch_offsets(lpsim_ctx *ctx, uint32_t n_scen, uint64_t *node_off, uint64_t *edge_off, uint64_t *cell_off,
                        uint64_t *trip_off);

/* ---- checkpoint and launch tuning -------------------------------------
 * lpsim_snapshot copies the whole simulation state (lane maps, vehicles,
 * queues, statistics, step) into device memory held by the context;
 * lpsim_restore returns to it.  Stepping after a restore gives exactly the
 * results of stepping from the snapshot the first time. */
int lpsim_snapshot(lpsim_ctx *ctx);
int lpsim_restore(lpsim_ctx *ctx);

typedef struct lpsim_tune_result {
    uint32_t block_size, blocks_per_sm, sort_period, chunk_steps; /* chosen (now in use) */
    double best_ms;     /* wall time of the chosen configuration over the window */
    double default_ms;  /* wall time of the configuration in use before tuning */
    uint32_t n_tried;
} lpsim_tune_result;

/* Autotuner: from the current state, run window_steps steps under each
 * candidate launch configuration (block size 128/256/512, 2/4/6 resident
 * 256-thread blocks per SM, sort period 64/128/256), restoring a snapshot
 * before each, and keep the fastest.  The context is left at the starting
 * state with the chosen configuration.  Results never depend on the
 * configuration, only speed does.  Best called at step 0 or at a multiple of
 * the chunk length. */
int lpsim_autotune(lpsim_ctx *ctx, uint32_t window_steps, lpsim_tune_result *out);

/* Set the launch configuration directly (e.g. from a stored tuning result). */
int lpsim_set_config(lpsim_ctx *ctx, uint32_t block_size, uint32_t blocks_per_sm, uint32_t sort_period,
                     uint32_t chunk_steps);

/* Per-kernel timing.  While on, each launch of the step kernels (step_p1:
 * car following, edge-end decisions, lane-change intents, departure and
 * entry claims; step_p2: entry conflicts, departures, lane changes), of the
 * compaction/sort sequence and of the light-load kernel stamps its own span
 * on the device: the GPU global timer when its first block starts working
 * (after the previous kernel's results are visible) and when its last block
 * ends.  One small kernel per graph chunk adds the spans up.  Nothing is
 * inserted between the kernels, so the CUDA graphs keep their programmatic
 * dependent launches and the light-load kernel still runs; spans of
 * consecutive kernels do not overlap, so their sum never exceeds the wall
 * time of the steps.  Switching on clears the sums; switching off keeps them
 * readable. */
int lpsim_set_kernel_timing(lpsim_ctx *ctx, int on);

typedef struct lpsim_kernel_times {
    double ms[4];           /* summed spans, ms: step_p1, step_p2, compaction + sort, light-load kernel */
    uint64_t launches[4];   /* launches timed, same order */
    uint64_t p1_veh_steps;  /* vehicle-steps handled by the timed step_p1 launches */
} lpsim_kernel_times;

/* Sums since timing was last switched on (zeros if it never was). */
int lpsim_get_kernel_times(lpsim_ctx *ctx, lpsim_kernel_times *out);

/* Largest trip count lpsim_get_state_noalloc serves: its scratch is a fixed
 * device array of LPSIM_NOALLOC_MAX_VEHICLES * 17 bytes (17 MiB). */
#define LPSIM_NOALLOC_MAX_VEHICLES 1048576u

/* lpsim_get_state without allocating anything.  The paper has no
 * counterpart: this is a service entry point of this library.
 *
 * lpsim_get_state takes device scratch for the call from cudaMalloc or the
 * allocator callback.  Callers that cannot allocate at that moment -- an
 * application whose device memory is a fixed pool already handed out, a
 * service capped at a device-memory budget it must not exceed while
 * running, or a host that installed no allocator and must not touch
 * cudaMalloc -- use this variant instead.  Its scratch is one file-scope
 * device array of the size above, which every GPU that loads the library
 * holds until the process exits.  The call makes no cudaMalloc, cudaFree or
 * allocator call: it clears the array, runs the same gather kernel on the
 * context's stream and copies into the caller's host buffers (same layout
 * and NULL rules as lpsim_get_state).
 *
 * n above LPSIM_NOALLOC_MAX_VEHICLES gives LPSIM_E_INVALID_ARG (use
 * lpsim_get_state).  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress, with that device current), and so does the
 * first call after the device's context was replaced (cudaDeviceReset); make
 * those first calls before any stream capture on the device.  Every call on a device
 * shares the one array and it keeps the last call's contents (the call
 * clears it before use): calls whose work overlaps on the GPU -- two
 * contexts on different streams, or two threads -- race on it and must be
 * serialised by the caller. */
int lpsim_get_state_noalloc(lpsim_ctx *ctx, uint64_t n, float *x, float *v, uint32_t *edge, uint8_t *lane,
                            uint32_t *route_idx, uint8_t *status);

/* Release every device and host resource of the context (NULL is a no-op). */
void lpsim_destroy(lpsim_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
