// Internal device-side layout shared by the translation units of liblpsim.
// Not part of the public ABI (include/lpsim.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lpsim {

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint8_t kEmpty = 0xFFu;
constexpr uint8_t kNoLane = 0xFFu;

// slot life cycle
constexpr uint8_t kLive = 0;
constexpr uint8_t kArrivedPending = 1;  // arrived this step: its cell is erased next step
constexpr uint8_t kDead = 2;

// trip status (public)
constexpr uint8_t kWaiting = 0;
constexpr uint8_t kActive = 1;
constexpr uint8_t kArrived = 2;

// light-load mode: one block of kSmallBlock threads runs a whole chunk when at
// most kSmallMax trips (the default of lpsim_params.light_trips) can be on the
// network or waiting during it
constexpr int kSmallBlock = 1024;
constexpr uint32_t kSmallMax = 1536;

// device error bits
constexpr uint32_t kErrCellTaken = 1u;   // a lane-map cell written twice in one step
constexpr uint32_t kErrSlotOverflow = 2u;

// Edge record: one 16-byte load gives everything the car-following part needs.
// Lane l, cell c of edge e lives at map[moff + l * stride(len) + c], stride =
// len rounded up to 16 bytes so every lane row starts 16-byte aligned.
struct __align__(16) EdgeRec {
    uint32_t moff;   // lane-map byte offset of lane 0
    uint16_t len;    // cells per lane
    uint8_t lanes;   // 1..4
    uint8_t arank;   // signal phase at the downstream node
    float v0;        // speed limit (free-flow speed)
    uint32_t dst;    // downstream node
};

struct __align__(8) NodeRec {
    uint32_t green;  // green steps per phase (0 = uncontrolled)
    uint8_t nphase;  // phases (1 + largest approach rank)
    uint8_t nout;    // outgoing edges
    uint16_t pad;
};

__host__ __device__ inline uint32_t row_stride(uint32_t len) { return (len + 15u) & ~15u; }

struct Model {
    float dt, a, s0, T, two_sqrt_ab, x0, g_a, g_b, alpha_i, alpha_a, alpha_b, eps_amp;
    uint64_t seed;
    uint32_t bin_steps, n_bins;
    float dlc_prob, dlc_gain;  // discretionary lane change (dlc_prob = 0: off)
};

// Vehicle type: its car-following parameters and top speed (free-flow speed
// on an edge = min(edge limit, vmax)).
constexpr uint32_t kMaxTypes = 8;
struct __align__(32) TypeRec {
    float a, s0, T, two_sqrt_ab, vmax, pad[3];
};

// Per route position q (the edge E = route[q] of some trip): the signal at
// E's downstream node (green steps and phase count of the node, E's phase)
// and the target lane on E for the movement onto route[q+1] (kNoLane when q
// is the trip's last position).  Precomputed on the device at load time so a
// vehicle entering an edge copies what the next edge's end needs.  (Eight
// bytes: four consecutive positions of a route share a 32-byte sector, so a
// vehicle finds the next position's record in L2 more often than not; adding
// the edge's speed limit and claim slot, tables that stay in L2 anyway, made
// the step slower.)
struct __align__(8) RouteRec {
    uint32_t green;
    uint8_t nphase, arank, tl, pad;
};

// One trip of a departure queue: vehicle id, departure step, route start and
// end positions.
struct __align__(16) QRec {
    uint32_t h, dep, r0, r1;
};

// What a vehicle copies when it enters an edge, plus its lane row (which a
// lane change moves): one 32-byte record per slot, read with two 16-byte
// loads and rewritten on entry with two 16-byte stores into one sector.  It
// holds the next edge's lane-map row geometry too, so a vehicle that may
// reach the stop line reads the entry cells of the next edge in the same
// round trip as its own leader scan.
struct __align__(32) EdgeState {
    uint32_t base;     // lane-map offset of cell 0 of the current lane
    uint32_t rpos;     // route position of the current edge (the edge is route[rpos])
    uint32_t en;       // next edge of the route, kNone on the last edge
    uint32_t sg;       // green steps of the signal at the end of the current edge (0 = none)
    float v0;          // speed limit of the current edge
    uint32_t nmoff;    // lane-map offset of lane 0 of the next edge (0 on the last edge)
    uint16_t len;      // cells per lane of the current edge
    uint16_t sph;      // phases of that signal | phase of the current edge << 8
    uint16_t nlen;     // cells per lane of the next edge
    uint8_t nlanes;    // lanes of the next edge
    uint8_t vt;        // vehicle type (Algorithm 1 State: V, recorded on every new edge)
};

__device__ __forceinline__ EdgeState load_es(const EdgeState *p) {
    const uint4 a = reinterpret_cast<const uint4 *>(p)[0], b = reinterpret_cast<const uint4 *>(p)[1];
    EdgeState r;
    r.base = a.x;
    r.rpos = a.y;
    r.en = a.z;
    r.sg = a.w;
    r.v0 = __uint_as_float(b.x);
    r.nmoff = b.y;
    r.len = (uint16_t)(b.z & 0xFFFFu);
    r.sph = (uint16_t)(b.z >> 16);
    r.nlen = (uint16_t)(b.w & 0xFFFFu);
    r.nlanes = (uint8_t)((b.w >> 16) & 0xFFu);
    r.vt = (uint8_t)(b.w >> 24);
    return r;
}

__device__ __forceinline__ void store_es(EdgeState *p, const EdgeState &r) {
    reinterpret_cast<uint4 *>(p)[0] = make_uint4(r.base, r.rpos, r.en, r.sg);
    reinterpret_cast<uint4 *>(p)[1] = make_uint4(__float_as_uint(r.v0), r.nmoff,
                                                 (uint32_t)r.len | ((uint32_t)r.sph << 16),
                                                 (uint32_t)r.nlen | ((uint32_t)r.nlanes << 16) |
                                                     ((uint32_t)r.vt << 24));
}

// Vehicle slots.  x and v are double-buffered by step parity: step k reads
// x[k&1] and writes x[(k+1)&1].  What the vehicle needs from its current edge
// (lane-row offset, length, speed limit, the signal at its end, the next edge
// of the route) is copied into its EdgeState when it enters the edge, so the
// common path reads the slot and the map only, and a crossing reads one edge
// record more.
struct Slots {
    EdgeState *es;
    // persistent
    uint32_t *id, *rlast;
    uint32_t *tent;    // step the vehicle entered its current edge
    uint32_t *pcell;   // cell of the previous step (erased this step), kNone
    uint32_t *imark;   // intent mark of the previous step (cleared this step), kNone
    uint32_t *cprev;   // claim slot won at the previous step (reset this step), kNone
    uint8_t *lane, *flag;
    uint8_t *tlc;      // target lane of the movement after the current edge (kNoLane on the last edge)
    float *x[2], *v[2];
};

// What step_p2 needs of a vehicle that asked to enter its next edge, packed
// by step_p1 at the vehicle's position in the crossing list so that step_p2
// reads it with four 16-byte loads instead of gathering slot fields.
struct __align__(16) CrossRec {
    uint32_t s, id, cslot, e;         // slot, vehicle, claim slot, current edge
    uint32_t en, rpos, tent, base;    // next edge, route position, entry step, current lane row
    uint32_t nbase, nen, nsg;         // on the next edge: lane row, the edge after, its signal's green
    float x, vn, nv0;                 // position and speed now, next edge's speed limit
    uint16_t len, nlen, nsph;         // current / next edge length, next signal phases | phase << 8
    uint8_t lane, tln;                // lane asked for | vehicle type << 2, target lane on the next edge
};

// What step_p2 needs of a departure request (packed by step_p1 for the queue
// head of an origin edge that asked to enter).
struct __align__(16) DepRec {
    uint32_t j, slot, h, r0;          // origin, claim slot, vehicle, route start
    uint32_t r1, qoff, qhead, qend;   // route end; the origin's queue records and head position
    uint32_t base, e0, nen, nsg;      // lane row asked for, origin edge, the edge after it, its signal's green
    float v0;                         // speed limit of the origin edge
    uint16_t len, nsph;               // origin edge length, signal phases | phase << 8
    uint8_t lane, tlc;                // lane asked for, target lane for the movement after the origin edge
    uint8_t vt;                       // vehicle type
};

// What step_p2 needs of a lane-change intender (packed by step_p1).
struct __align__(16) IntendRec {
    uint32_t s, base;                 // slot, current lane row
    uint64_t hk;                      // lane-change draw key
    float x, xn, vn;                  // position now and next, speed next
    uint16_t len;
    uint8_t lane, up;
};

struct Dev {
    // network
    const EdgeRec *edge;
    const NodeRec *node;
    const uint32_t *slot_off;  // first (edge, lane) claim slot of each edge
    const uint8_t *orank;      // rank of the edge among the out-edges of its source
    uint8_t *map[3];           // lane maps, step k reads map[k%3], writes map[(k+1)%3]
    uint8_t *imap[2];          // lane-change intent marks of step k: imap[k&1]
    uint32_t *claim[2];        // per (edge, lane): lowest id asking to enter, by step parity
    // trips, by vehicle id
    const uint32_t *route;     // all routes, vehicle-id order
    const uint32_t *roff;      // route start of vehicle id (n + 1 entries)
    const RouteRec *rrec;      // per route position
    const uint64_t *hkey;      // lane-change draw key: scenario seed ^ scenario-local id * C1
    const TypeRec *types;      // vehicle types (typed != 0)
    const uint8_t *trip_vt;    // vehicle type by id (typed != 0)
    uint32_t typed;            // 0: every vehicle has the run parameters and no top speed of its own
    uint32_t hkey_from_id;     // 1: one scenario, whose key is m.seed ^ id * C1 (no load needed)
    uint32_t *dep_act, *arr;
    uint8_t *status;
    // departure queues, one per origin edge (queue records in queue order)
    uint32_t n_org;
    const uint32_t *org_edge, *org_qoff, *org_qend;
    const EdgeRec *org_rec;    // edge record of each origin edge
    const QRec *qrec;
    uint32_t *org_head;        // position of the head in its queue
    QRec *org_hd;              // head record (h = kNone: queue empty)
    uint32_t *dprev;           // claim slot won at the previous step (kNone)
    // slots (current set: the host alternates two sets around each compaction)
    Slots s;
    uint32_t cap;              // slot capacity
    // per-step lists, by step parity
    CrossRec *cross_list[2];
    IntendRec *intend_list[2];
    uint32_t *counts;          // [0..1] cross count by parity, [2..3] intend count, [4..5] departure requests,
                               // [6..7] stop-line intents (at the top of intend_list)
    DepRec *dep_rec[2];        // departure requests, by parity
    // crossings of the current chunk (or direct step), applied to the link
    // statistics by one kernel at its end instead of seven scattered atomics
    // per crossing inside step_p2: {edge left, edge entered, step the edge
    // left was entered, step} or {kNone, ...} for a crossing request that lost.
    // *ev_n entries so far; past ev_cap the crossings update the counters
    // directly.
    uint4 *ev_log;
    uint32_t ev_cap;
    uint32_t *ev_n;
    // {*n_slots, *ev_n} at the start of the current step (written by
    // step_P1, read by step_P2, which advances the two live values)
    uint32_t *snap;
    // per lane row (index = the row's map offset / 16): the crossing request
    // made from it at step k, {k, claim slot, vehicle id, 0}; a stop-line
    // lane-change intent reads the row it aims at to learn whether a hold
    // will land on its target cell in the same kernel
    uint4 *xreq;
    // statistics; binned arrays are bin-major ([bin][edge]) so the updates of
    // one step fall in one or two rows that stay in L2
    unsigned long long *ent, *ext, *tts;
    uint32_t *bin_in, *bin_tt, *bin_cnt, *bin_occ;
    uint32_t n_edges;
    // run state
    uint32_t *kbase;           // step of the first step of the current graph chunk
    uint32_t *n_slots;         // slots in use
    unsigned long long *ctr;   // [0] veh_steps, [1] arrived, [2] lane changes, [3] crossings + departures,
                               // [4] departed
    uint32_t *err;
    uint32_t check;            // 1: verify every next-map write lands on an empty cell
    // Kernel timing (nullptr when off): per step koff of a chunk, the span of
    // each phase as {~first block start, last block end} in %globaltimer
    // nanoseconds -- tspan[6 koff + 2 ph], ph 0 step_p1, 1 step_p2, 2 the
    // compaction sequence -- and {~start, end} of the light-load kernel at
    // tspan[6 C]; the start is stored inverted so that atomicMax over a
    // zeroed slot keeps the earliest.  timing_fold adds the spans into
    // tacc: [0..3] ns of step_p1, step_p2, compaction, light-load kernel,
    // [4..7] their launches, [8] vehicle-steps handled by step_p1.
    unsigned long long *tspan, *tacc;
    uint32_t tspan_light;      // index of the light-load kernel's pair (6 C)
    Model m;
};

// %globaltimer (nanoseconds, one clock for the whole GPU)
__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Start and end stamps of a kernel's span in slot pair `pair` (timing only;
// one thread per block; the end stamp after a block barrier, so the block's
// last thread has finished).
__device__ __forceinline__ void span_start(const Dev &d, uint32_t pair) {
    if (d.tspan && threadIdx.x == 0) atomicMax(&d.tspan[2 * pair], ~gtime());
}
__device__ __forceinline__ void span_end(const Dev &d, uint32_t pair) {
    if (d.tspan) {
        __syncthreads();
        if (threadIdx.x == 0) atomicMax(&d.tspan[2 * pair + 1], gtime());
    }
}

// kernels of a step; koff = offset of this step inside the chunk (step k =
// *kbase + koff); kph = any number congruent to k modulo 6, known when the
// launch is recorded (koff inside a graph chunk, whose first step is a
// multiple of 6; k itself for a direct launch), so the kernels pick the
// parity buffers and the rotating lane maps without waiting for *kbase
void launch_phase(const Dev &d, int phase, uint32_t koff, uint32_t kph, int grid, int block, cudaStream_t st);
void launch_chunk_end(const Dev &d, uint32_t steps, cudaStream_t st);
// the logged crossings of the chunk into the link statistics (before chunk_end)
void launch_apply_crossings(const Dev &d, int grid, cudaStream_t st);
// kernel timing: the spans of steps [0, nsteps) of the chunk (and of the
// light-load kernel) into the accumulators; clears the span slots
void launch_timing_fold(const Dev &d, uint32_t nsteps, cudaStream_t st);
// steps [k0, k0 + nsteps) in one block (light load); olist: n_org scratch
// entries, no: one device counter
// shared memory the light-load kernel may take for the lane maps (five maps)
constexpr size_t kSmallMapSmem = 200 * 1024;
cudaError_t launch_small(const Dev &d, uint32_t k0, uint32_t nsteps, uint32_t *olist, uint32_t *no,
                         uint32_t map_words, cudaStream_t st);

// compaction (and optional sort by lane-map cell) of the slots after step k;
// src/dst slot sets; writes *n_slots
struct SortWork {
    uint32_t *tile_cnt, *tile_off;   // per tile
    uint32_t *key[2], *perm[2];      // radix sort ping-pong
    uint32_t *hist;                  // 256 digits x tiles
    uint32_t max_tiles;
    uint32_t key_bits;
};
// returns the number of kernels launched
int launch_compact(const Dev &d, const Slots &dst, const SortWork &w, uint32_t koff, bool sort, int grid,
                   cudaStream_t st);
uint32_t compact_tile();

// per-route-position records (load time)
void launch_route_records(const Dev &d, uint64_t n_trips, RouteRec *out, cudaStream_t st);
void launch_transpose_bins(const uint32_t *in, uint32_t n_edges, uint32_t n_bins, uint32_t *out, cudaStream_t st);

// helpers for the query functions
void launch_state_scatter(const Dev &d, uint32_t k, float *x, float *v, uint32_t *edge, uint8_t *lane,
                          uint32_t *ridx, cudaStream_t st);
void launch_max_arrival(const Dev &d, uint64_t n, uint32_t *out, cudaStream_t st);

}  // namespace lpsim
