/*
 * lpsim_oracle.c -- single-threaded CPU oracle of the per-step vehicle update
 * (Algorithm 1, Sec. 3.1-3.2 of arXiv 2406.08496).
 *
 * TEST INFRASTRUCTURE ONLY: the GPU library is checked against this file; the
 * product path never loads it.  Build with -O2 -ffp-contract=off and no
 * fast-math so every float operation is a separately rounded IEEE binary32
 * operation in the order written.
 *
 * Model and readings (the paper names the rules but not their formulas):
 *
 *  Lane map (Sec. 3.1): one byte per metre of lane; 255 = empty, 0..254 = the
 *    occupying vehicle's speed in m/s, truncated.  An edge of length L metres
 *    has len = max(1, ceil(L)) cells per lane and the dynamics use
 *    L_e = (float)len.  Two maps: M_cur holds step k, M_nxt receives step k+1.
 *
 *  Vehicle ids: rank of the trip after a stable sort by departure step (the
 *    paper sorts trips by departure time, Sec. 4 / Table 6).
 *
 *  Step k, computed for every vehicle from the state at k only (Jacobi update,
 *  eq. vehicle_dynamics):
 *   P1 leader     nearest occupied cell c_f > floor(x) in the own lane of the
 *                 own edge (the next edge is only looked at when crossing,
 *                 Sec. 3.1 Remark, Intersection Modeling).
 *      speed      if the leader is within d_front = 2*dt*v (Algorithm 1) the
 *                 IDM (eq. Car Following, Treiber's form with delta = 4):
 *                   s_star = s0 + max(0, v*T + v*(v - v_f)/(2 sqrt(a b)))
 *                   acc = a*(1 - (v/v0)^4 - (s_star/s)^2),  v' = max(0, v + acc*dt)
 *                 else v' = v_free = the edge speed limit (Algorithm 1).
 *      types      (Algorithm 1 State: vehicle type V; multimodal, Sec. 5)
 *                 a vehicle of type t uses the type's a, b, s0, T above and
 *                 v0 = v_free = min(edge limit, vmax_t); type 0 defaults to
 *                 the run parameters and vmax 254.
 *      move       x' = x + v'*dt; no-crash clamp (Sec. 3.1 Remark: vehicles do
 *                 not crash): if x' > c_f - s0 then x' = max(x, c_f - s0), v' = 0.
 *      edge end   x' >= L_e: on the last route edge the vehicle arrives; else,
 *                 if the signal is green, it asks for cell 0 of the next edge
 *                 (Sec. 3.2: a vehicle moves on only if the first byte of the
 *                 downstream edge is free); else it waits at the stop line.
 *      signals    node with G > 0 green steps whose approaches carry phase ranks
 *                 0..n-1 (n = 1 + the largest rank; by default every approach
 *                 is its own phase, ranked by edge id): an approach of rank j
 *                 is green iff (k / G) mod n == j.
 *      lane change (eq. Lane Change) target lane for the next movement
 *                 tl = rank(next edge among out-edges of the node) * lanes / n_out;
 *                 a vehicle off tl moves one lane toward it; upward moves only
 *                 on odd k, downward only on even k; probability
 *                 m = 1 - (L_e - x)/x0 when L_e - x < x0, else 0; draw
 *                 u = top 24 bits of SplitMix64(seed ^ id*C1 ^ k*C2) / 2^24.
 *      discretionary lane change (an extension: the paper names only the
 *                 mandatory change; off when dlc_prob = 0): a staying vehicle
 *                 outside the mandatory case above (no next movement, already
 *                 in its target lane, or farther than x0 from the end) held
 *                 below its free speed by its leader c_f (v' < v0: the IDM or
 *                 the clamp acted) with that leader slower than its free speed
 *                 (speed byte < v0) intends one lane up on odd k, down on even
 *                 k (if that lane exists) when, in that lane of M_cur, the
 *                 nearest occupied cell c_a in [floor(x), floor(x)+63] is
 *                 absent or c_a - c_f >= dlc_gain, and u < dlc_prob (the same
 *                 draw u); P3 then judges it like any intent.
 *      departure  the lowest-id waiting vehicle of each first edge whose
 *                 departure step has come asks for cell 0 of that edge.
 *      entry lane lanes of the entered edge ordered by distance to its own tl
 *                 (ties to the lower index); the first one whose cell 0 is
 *                 empty in M_cur is requested, none -> wait.
 *      conflicts  several requests for one (edge, lane): the lowest vehicle id
 *                 wins (the paper resolves this with an atomic, Sec. 3.1 Remark).
 *   P2 M_nxt      stayers write their cell; winners enter at x = 0 (crossers
 *                 keep v', departures start at v = 0); losers and red-held
 *                 vehicles stop at max(x, L_e - 1) with v = 0.
 *   P3 gaps       (eq. Gap Acceptance) in the target lane of M_cur, lead = nearest
 *                 occupied cell in [floor(x), floor(x)+63], lag = nearest in
 *                 [floor(x)-64, floor(x)-1];
 *                   G_lead = g_a + max(0, alpha_i v' - alpha_a v_a) + eps_a
 *                   G_lag  = g_b + max(0, alpha_b v_b - alpha_i v') + eps_b
 *                 accept iff c_a - x' >= G_lead, x' - c_b >= G_lag, floor(x') >= 1
 *                 and the target cell is empty in M_nxt after P2.
 *   P4            accepted changers move their M_nxt byte sideways; every
 *                 vehicle's step-k cell is erased from M_cur; the maps swap.
 */
#include "lpsim_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { ST_WAITING = 0, ST_ACTIVE = 1, ST_ARRIVED = 2 };
enum { ACT_NONE = 0, ACT_STAY, ACT_INTEND, ACT_HOLD, ACT_CROSS, ACT_ARRIVE };
#define EMPTY 255u
#define NO_CLAIM 0xFFFFFFFFu

typedef struct {
    float a, s0, T, two_sqrt_ab, vmax;
} vtype_rec;

struct orc_sim {
    orc_params p;
    float two_sqrt_ab;
    vtype_rec types[ORC_MAX_TYPES];
    uint32_t n_types;
    uint8_t *vt;                /* vehicle type, by id */
    /* network */
    uint32_t n_nodes, n_edges;
    uint32_t *src, *dst, *len, *green, *n_in, *n_out, *n_phase;
    float *v0;
    uint8_t *lanes, *arank, *orank;
    uint64_t *moff, mcells;     /* lane-map offset of each edge, total cells */
    uint64_t *slot_off;         /* first (edge, lane) slot of each edge */
    uint8_t *Mcur, *Mnxt;
    /* demand */
    int loaded;
    uint64_t n;
    uint32_t *dep;
    uint64_t *roff;
    uint32_t *redge;
    /* vehicles, by id */
    uint8_t *status, *lane, *act, *tlane, *accept;
    int8_t *dir;
    uint32_t *e, *r, *t_enter, *dep_act, *arr;
    float *x, *v, *xn, *vn;
    uint64_t *old_cell;
    /* active vehicles (any order; every rule is order independent) */
    uint32_t *active, n_active_list, *next_active;
    /* departure queues: ids with route[0] == e, ascending */
    uint64_t *qoff, *qhead;
    uint32_t *qid;
    uint32_t *pending, n_pending; /* edges whose queue head may depart */
    uint8_t *is_pending;
    uint64_t released;            /* ids < released have depart_step <= k */
    uint8_t *dreq;                /* requested lane per pending edge (EMPTY = none) */
    /* claims */
    uint32_t *claim;
    /* statistics */
    uint64_t *ent, *ext, *tts;
    uint32_t *bin_in, *bin_tt, *bin_cnt, *bin_occ;
    /* counters */
    uint32_t k;
    uint64_t veh_steps, n_arrived, n_lane_changes;
};

/* ---------------------------------------------------------------- helpers */

static uint64_t splitmix64_mix(uint64_t z) {
    /* SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014) */
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static float unit24(uint64_t h) { return (float)(h >> 40) * (1.0f / 16777216.0f); }

static uint8_t speed_byte(float v) {
    float t = v < 254.0f ? v : 254.0f;
    return (uint8_t)t;
}

static float fmax0(float t) { return t > 0.0f ? t : 0.0f; }

static uint64_t cell_index(const orc_sim *s, uint32_t e, uint32_t ln, uint32_t c) {
    return s->moff[e] + (uint64_t)ln * s->len[e] + c;
}

static int is_green(const orc_sim *s, uint32_t e, uint32_t k) {
    uint32_t node = s->dst[e];
    uint32_t G = s->green[node];
    if (G == 0) return 1;
    return (k / G) % s->n_phase[node] == s->arank[e];
}

/* Target lane on edge `edge` for the movement onto `next` (Lane Change reading). */
static uint32_t target_lane(const orc_sim *s, uint32_t edge, uint32_t next) {
    return ((uint32_t)s->orank[next] * s->lanes[edge]) / s->n_out[s->dst[edge]];
}

/* Lane in which a vehicle entering route position q of trip `id` asks for
 * cell 0, or EMPTY when every lane's cell 0 is taken in M_cur. */
static uint32_t entry_lane(const orc_sim *s, uint32_t id, uint64_t q) {
    uint64_t first = s->roff[id], last = s->roff[id + 1] - 1;
    uint32_t en = s->redge[first + q];
    uint32_t nl = s->lanes[en];
    uint32_t tl = (first + q < last) ? target_lane(s, en, s->redge[first + q + 1]) : 0;
    for (uint32_t d = 0; d < nl; d++) {
        if (tl >= d && s->Mcur[cell_index(s, en, tl - d, 0)] == EMPTY) return tl - d;
        if (d > 0 && tl + d < nl && s->Mcur[cell_index(s, en, tl + d, 0)] == EMPTY) return tl + d;
    }
    return EMPTY;
}

/* the IDM branch for a vehicle of type y: speed v, leader byte speed vf,
 * gap s, free-flow speed v0 */
static float idm_speed_type(const vtype_rec *y, float dt, float v, float vf, float s, float v0) {
    float dv = v - vf;
    float z = v * y->T + (v * dv) / y->two_sqrt_ab;
    float s_star = y->s0 + fmax0(z);
    float r = v / v0;
    float q = s_star / s;
    float acc = y->a * ((1.0f - (r * r) * (r * r)) - q * q);
    return fmax0(v + acc * dt);
}

float orc_idm_speed(const orc_params *p, float v, float vf, float s, float v0) {
    vtype_rec y;
    y.a = p->a;
    y.s0 = p->s0;
    y.T = p->T;
    y.two_sqrt_ab = (float)(2.0 * sqrt((double)p->a * (double)p->b));
    y.vmax = 254.0f;
    return idm_speed_type(&y, p->dt, v, vf, s, v0);
}

static int put(orc_sim *s, uint64_t idx, uint8_t val) {
    if (s->Mnxt[idx] != EMPTY) return -7; /* two vehicles in one cell */
    s->Mnxt[idx] = val;
    return 0;
}

static void stat_entry(orc_sim *s, uint32_t e, uint32_t k) {
    s->ent[e]++;
    if (s->p.bin_steps) {
        uint32_t b = (k + 1) / s->p.bin_steps;
        if (b < s->p.n_bins) s->bin_in[(uint64_t)e * s->p.n_bins + b]++;
    }
}

static void stat_exit(orc_sim *s, uint32_t e, uint32_t k, uint32_t t_enter) {
    uint32_t steps = k + 1 - t_enter;
    s->ext[e]++;
    s->tts[e] += steps;
    if (s->p.bin_steps) {
        uint32_t b = t_enter / s->p.bin_steps;
        if (b < s->p.n_bins) {
            s->bin_tt[(uint64_t)e * s->p.n_bins + b] += steps;
            s->bin_cnt[(uint64_t)e * s->p.n_bins + b]++;
        }
    }
}

/* ------------------------------------------------------------ construction */

#define XALLOC(ptr, count) do { (ptr) = calloc((size_t)(count) + 1, sizeof(*(ptr))); if (!(ptr)) return -2; } while (0)

int orc_create(orc_sim **out, uint32_t n_nodes, uint32_t n_edges, const uint32_t *src, const uint32_t *dst,
               const float *len_m, const uint8_t *lanes, const float *vmax, const uint32_t *green_steps,
               const uint8_t *approach_rank, const orc_params *p) {
    if (!out || !src || !dst || !len_m || !lanes || !vmax || !green_steps || !p) return -1;
    if (n_nodes == 0 || n_edges == 0) return -1;
    if (!(p->dt > 0.0f) || !(p->a > 0.0f) || !(p->b > 0.0f) || !(p->s0 >= 0.0f) || !(p->x0 > 0.0f)) return -1;
    if (!(p->dlc_prob >= 0.0f && p->dlc_prob <= 1.0f) || !(p->dlc_gain >= 0.0f)) return -1;
    if (p->bin_steps == 0 && p->n_bins != 0) return -1;
    for (uint32_t e = 0; e < n_edges; e++) {
        if (src[e] >= n_nodes || dst[e] >= n_nodes) return -1;
        if (lanes[e] < 1 || lanes[e] > 4) return -1;
        if (!(len_m[e] > 0.0f) || !(len_m[e] <= 65535.0f)) return -1;
        if (!(vmax[e] > 0.0f) || !(vmax[e] <= 254.0f)) return -1;
    }
    orc_sim *s = calloc(1, sizeof(orc_sim));
    if (!s) return -2;
    *out = s;
    s->p = *p;
    s->two_sqrt_ab = (float)(2.0 * sqrt((double)p->a * (double)p->b));
    s->n_types = 1;
    s->types[0].a = p->a;
    s->types[0].s0 = p->s0;
    s->types[0].T = p->T;
    s->types[0].two_sqrt_ab = s->two_sqrt_ab;
    s->types[0].vmax = 254.0f;
    s->n_nodes = n_nodes;
    s->n_edges = n_edges;
    XALLOC(s->src, n_edges); XALLOC(s->dst, n_edges); XALLOC(s->len, n_edges); XALLOC(s->v0, n_edges);
    XALLOC(s->lanes, n_edges); XALLOC(s->arank, n_edges); XALLOC(s->orank, n_edges);
    XALLOC(s->green, n_nodes); XALLOC(s->n_in, n_nodes); XALLOC(s->n_out, n_nodes); XALLOC(s->n_phase, n_nodes);
    XALLOC(s->moff, n_edges); XALLOC(s->slot_off, n_edges);
    uint64_t cells = 0, slots = 0;
    for (uint32_t e = 0; e < n_edges; e++) {
        s->src[e] = src[e];
        s->dst[e] = dst[e];
        uint32_t c = (uint32_t)ceilf(len_m[e]);
        s->len[e] = c < 1 ? 1 : c;
        s->v0[e] = vmax[e];
        s->lanes[e] = lanes[e];
        s->moff[e] = cells;
        cells += (uint64_t)s->len[e] * lanes[e];
        s->slot_off[e] = slots;
        slots += lanes[e];
    }
    s->mcells = cells;
    for (uint32_t i = 0; i < n_nodes; i++) s->green[i] = green_steps[i];
    /* approach rank: given, or rank among incoming edges of dst by edge id;
     * out rank: rank among outgoing edges of src by edge id */
    for (uint32_t e = 0; e < n_edges; e++) {
        s->orank[e] = (uint8_t)s->n_out[src[e]];
        s->n_out[src[e]]++;
        if (s->n_out[src[e]] > 255) return -1;
        uint32_t rank = s->n_in[dst[e]]++;
        if (s->n_in[dst[e]] > 255) return -1;
        s->arank[e] = approach_rank ? approach_rank[e] : (uint8_t)rank;
    }
    for (uint32_t e = 0; e < n_edges; e++) {
        if (s->arank[e] >= s->n_in[dst[e]]) return -1;
        if (s->arank[e] + 1u > s->n_phase[dst[e]]) s->n_phase[dst[e]] = s->arank[e] + 1u;
    }
    XALLOC(s->Mcur, cells); XALLOC(s->Mnxt, cells);
    memset(s->Mcur, EMPTY, cells);
    memset(s->Mnxt, EMPTY, cells);
    XALLOC(s->claim, slots);
    for (uint64_t i = 0; i < slots; i++) s->claim[i] = NO_CLAIM;
    XALLOC(s->ent, n_edges); XALLOC(s->ext, n_edges); XALLOC(s->tts, n_edges);
    uint64_t nb = (uint64_t)n_edges * p->n_bins;
    XALLOC(s->bin_in, nb); XALLOC(s->bin_tt, nb); XALLOC(s->bin_cnt, nb); XALLOC(s->bin_occ, nb);
    return 0;
}

int orc_set_vehicle_types(orc_sim *s, uint32_t n_types, const orc_vehicle_type *types) {
    if (!s || !types || n_types == 0 || n_types > ORC_MAX_TYPES) return -1;
    if (s->loaded) return -4;
    for (uint32_t t = 0; t < n_types; t++) {
        const orc_vehicle_type *y = &types[t];
        if (!(y->a > 0.0f) || !(y->b > 0.0f) || !(y->s0 >= 0.0f) || !(y->T == y->T) || !(y->vmax > 0.0f) ||
            !(y->vmax <= 254.0f))
            return -1;
        s->types[t].a = y->a;
        s->types[t].s0 = y->s0;
        s->types[t].T = y->T;
        s->types[t].two_sqrt_ab = (float)(2.0 * sqrt((double)y->a * (double)y->b));
        s->types[t].vmax = y->vmax;
    }
    s->n_types = n_types;
    return 0;
}

int orc_load_demand(orc_sim *s, uint64_t n, const uint32_t *depart_step, const uint64_t *route_off,
                    const uint32_t *route_edges, uint32_t *out_vid) {
    return orc_load_demand_typed(s, n, depart_step, route_off, route_edges, NULL, out_vid);
}

int orc_load_demand_typed(orc_sim *s, uint64_t n, const uint32_t *depart_step, const uint64_t *route_off,
                          const uint32_t *route_edges, const uint8_t *vtype, uint32_t *out_vid) {
    if (!s || !depart_step || !route_off || !route_edges) return -1;
    if (s->loaded) return -4;
    if (n >= 0xFFFFFFFFull) return -1;
    if (route_off[0] != 0) return -1;
    if (vtype)
        for (uint64_t j = 0; j < n; j++)
            if (vtype[j] >= s->n_types) return -1;
    for (uint64_t j = 0; j < n; j++) {
        if (route_off[j + 1] <= route_off[j]) return -1; /* empty route */
        for (uint64_t q = route_off[j]; q < route_off[j + 1]; q++) {
            if (route_edges[q] >= s->n_edges) return -1;
            if (q > route_off[j] && s->dst[route_edges[q - 1]] != s->src[route_edges[q]]) return -1;
        }
    }
    /* stable sort of trips by departure step: counting sort on a copy */
    uint64_t *order = malloc((n + 1) * sizeof(uint64_t));
    if (!order) return -2;
    for (uint64_t j = 0; j < n; j++) order[j] = j;
    /* insertion-free stable sort: merge sort on keys */
    {
        uint64_t *tmp = malloc((n + 1) * sizeof(uint64_t));
        if (!tmp) { free(order); return -2; }
        for (uint64_t width = 1; width < n; width *= 2) {
            for (uint64_t lo = 0; lo < n; lo += 2 * width) {
                uint64_t mid = lo + width < n ? lo + width : n;
                uint64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
                uint64_t a = lo, b = mid, o = lo;
                while (a < mid && b < hi) {
                    if (depart_step[order[b]] < depart_step[order[a]]) tmp[o++] = order[b++];
                    else tmp[o++] = order[a++];
                }
                while (a < mid) tmp[o++] = order[a++];
                while (b < hi) tmp[o++] = order[b++];
            }
            memcpy(order, tmp, n * sizeof(uint64_t));
        }
        free(tmp);
    }
    s->n = n;
    XALLOC(s->dep, n); XALLOC(s->roff, n + 1); XALLOC(s->vt, n);
    uint64_t total = route_off[n];
    XALLOC(s->redge, total);
    s->roff[0] = 0;
    for (uint64_t id = 0; id < n; id++) {
        uint64_t j = order[id];
        s->dep[id] = depart_step[j];
        s->vt[id] = vtype ? vtype[j] : 0;
        uint64_t len = route_off[j + 1] - route_off[j];
        memcpy(s->redge + s->roff[id], route_edges + route_off[j], len * sizeof(uint32_t));
        s->roff[id + 1] = s->roff[id] + len;
        if (out_vid) out_vid[j] = (uint32_t)id;
    }
    free(order);
    XALLOC(s->status, n); XALLOC(s->lane, n); XALLOC(s->act, n); XALLOC(s->tlane, n); XALLOC(s->accept, n);
    XALLOC(s->dir, n); XALLOC(s->e, n); XALLOC(s->r, n); XALLOC(s->t_enter, n);
    XALLOC(s->dep_act, n); XALLOC(s->arr, n); XALLOC(s->x, n); XALLOC(s->v, n);
    XALLOC(s->xn, n); XALLOC(s->vn, n); XALLOC(s->old_cell, n);
    XALLOC(s->active, n); XALLOC(s->next_active, n);
    for (uint64_t id = 0; id < n; id++) { s->dep_act[id] = 0xFFFFFFFFu; s->arr[id] = 0xFFFFFFFFu; }
    /* departure queues */
    XALLOC(s->qoff, s->n_edges + 1); XALLOC(s->qhead, s->n_edges); XALLOC(s->qid, n);
    for (uint64_t id = 0; id < n; id++) s->qoff[s->redge[s->roff[id]] + 1]++;
    for (uint32_t e = 0; e < s->n_edges; e++) s->qoff[e + 1] += s->qoff[e];
    {
        uint64_t *fill = malloc(((size_t)s->n_edges + 1) * sizeof(uint64_t));
        if (!fill) return -2;
        memcpy(fill, s->qoff, (size_t)s->n_edges * sizeof(uint64_t));
        for (uint64_t id = 0; id < n; id++) s->qid[fill[s->redge[s->roff[id]]]++] = (uint32_t)id;
        free(fill);
    }
    XALLOC(s->pending, s->n_edges); XALLOC(s->is_pending, s->n_edges); XALLOC(s->dreq, s->n_edges);
    s->loaded = 1;
    return 0;
}

/* ------------------------------------------------------------------- step */

/* P1 for one active vehicle: speed, move, and what it does at the edge end. */
static void decide(orc_sim *s, uint32_t i, uint32_t k) {
    const orc_params *p = &s->p;
    uint32_t e = s->e[i], ln = s->lane[i], len = s->len[e];
    float x = s->x[i], v = s->v[i], L = (float)len;
    uint32_t c = (uint32_t)x;
    uint64_t base = cell_index(s, e, ln, 0);
    s->old_cell[i] = base + c;

    /* leader: nearest occupied cell ahead in the own lane of the own edge */
    int has_f = 0;
    uint32_t cf = 0;
    for (uint32_t q = c + 1; q < len; q++)
        if (s->Mcur[base + q] != EMPTY) { has_f = 1; cf = q; break; }

    /* the vehicle's type: its IDM parameters, and its free-flow speed on
     * this edge, the lower of the edge limit and the type's top speed */
    const vtype_rec *y = &s->types[s->vt[i]];
    float v0 = s->v0[e] < y->vmax ? s->v0[e] : y->vmax;
    float vn;
    float d_front = (2.0f * p->dt) * v;
    if (has_f && ((float)cf - x) <= d_front)
        vn = idm_speed_type(y, p->dt, v, (float)s->Mcur[base + cf], (float)cf - x, v0);
    else
        vn = v0;
    float xn = x + vn * p->dt;
    if (has_f) {
        float lim = (float)cf - y->s0;
        if (xn > lim) { xn = x > lim ? x : lim; vn = 0.0f; }
    }
    s->xn[i] = xn;
    s->vn[i] = vn;
    s->dir[i] = 0;

    uint64_t first = s->roff[i], last = s->roff[i + 1] - 1, pos = first + s->r[i];
    if (xn >= L) {
        if (pos == last) { s->act[i] = ACT_ARRIVE; return; }
        if (!is_green(s, e, k)) { s->act[i] = ACT_HOLD; return; }
        uint32_t l = entry_lane(s, i, s->r[i] + 1);
        if (l == EMPTY) { s->act[i] = ACT_HOLD; return; }
        s->act[i] = ACT_CROSS;
        s->tlane[i] = (uint8_t)l;
        return;
    }
    s->act[i] = ACT_STAY;
    if (s->lanes[e] < 2) return;
    int mandatory = 0;
    if (pos < last) {
        uint32_t tl = target_lane(s, e, s->redge[pos + 1]);
        if (tl != ln) {
            int dir = tl > ln ? 1 : -1;
            float xrem = L - x;
            mandatory = xrem < p->x0;
            if ((dir > 0) == ((k & 1u) == 1u)) {
                float m = xrem >= p->x0 ? 0.0f : 1.0f - xrem / p->x0;
                uint64_t h = splitmix64_mix(p->seed ^ ((uint64_t)i * 0x9E3779B97F4A7C15ULL) ^
                                            ((uint64_t)k * 0xD1B54A32D192ED03ULL));
                if (unit24(h) < m) { s->act[i] = ACT_INTEND; s->dir[i] = (int8_t)dir; }
            }
        }
    }
    /* discretionary lane change: held up by a slower leader, a longer gap
     * ahead in the lane of this step's direction */
    if (mandatory || !(p->dlc_prob > 0.0f)) return;
    if (!(has_f && vn < v0 && (float)s->Mcur[base + cf] < v0)) return;
    int dir = (k & 1u) ? 1 : -1;
    if (dir > 0 ? ln + 1 >= s->lanes[e] : ln == 0) return;
    uint64_t base2 = cell_index(s, e, (uint32_t)((int)ln + dir), 0);
    for (uint32_t q = c; q < len && q <= c + 63; q++)
        if (s->Mcur[base2 + q] != EMPTY) {
            if (!((float)q - (float)cf >= p->dlc_gain)) return;
            break;
        }
    uint64_t h = splitmix64_mix(p->seed ^ ((uint64_t)i * 0x9E3779B97F4A7C15ULL) ^ ((uint64_t)k * 0xD1B54A32D192ED03ULL));
    if (unit24(h) < p->dlc_prob) { s->act[i] = ACT_INTEND; s->dir[i] = (int8_t)dir; }
}

/* P3 for one lane-change intender: gap acceptance against M_cur, free target
 * cell against M_nxt as written by P2. */
static int gap_accept(const orc_sim *s, uint32_t i, uint32_t k) {
    const orc_params *p = &s->p;
    uint32_t e = s->e[i], len = s->len[e];
    uint32_t ln2 = (uint32_t)((int)s->lane[i] + s->dir[i]);
    uint64_t base2 = cell_index(s, e, ln2, 0);
    float x = s->x[i], xn = s->xn[i], vn = s->vn[i];
    uint32_t c0 = (uint32_t)x, cn = (uint32_t)xn;

    int has_a = 0, has_b = 0;
    uint32_t ca = 0, cb = 0;
    for (uint32_t q = c0; q < len && q <= c0 + 63; q++)
        if (s->Mcur[base2 + q] != EMPTY) { has_a = 1; ca = q; break; }
    for (uint32_t d = 1; d <= 64 && d <= c0; d++)
        if (s->Mcur[base2 + c0 - d] != EMPTY) { has_b = 1; cb = c0 - d; break; }

    float eps_a = 0.0f, eps_b = 0.0f;
    if (p->eps_amp > 0.0f) {
        uint64_t h = splitmix64_mix(p->seed ^ ((uint64_t)i * 0x9E3779B97F4A7C15ULL) ^
                                    ((uint64_t)k * 0xD1B54A32D192ED03ULL));
        eps_a = p->eps_amp * (2.0f * unit24(splitmix64_mix(h ^ 0x632BE59BD9B4E019ULL)) - 1.0f);
        eps_b = p->eps_amp * (2.0f * unit24(splitmix64_mix(h ^ 0x8CB92BA72F3D8DD7ULL)) - 1.0f);
    }
    if (has_a) {
        float va = (float)s->Mcur[base2 + ca];
        float G_lead = (p->g_a + fmax0(p->alpha_i * vn - p->alpha_a * va)) + eps_a;
        if (!(((float)ca - xn) >= G_lead)) return 0;
    }
    if (has_b) {
        float vb = (float)s->Mcur[base2 + cb];
        float G_lag = (p->g_b + fmax0(p->alpha_b * vb - p->alpha_i * vn)) + eps_b;
        if (!((xn - (float)cb) >= G_lag)) return 0;
    }
    if (cn < 1) return 0;
    return s->Mnxt[base2 + cn] == EMPTY;
}

static int step_once(orc_sim *s) {
    uint32_t k = s->k;
    const orc_params *p = &s->p;
    int rc;

    /* release trips whose departure step has come; their first edge may now have a ready head */
    while (s->released < s->n && s->dep[s->released] <= k) {
        uint32_t id = (uint32_t)s->released++;
        uint32_t e0 = s->redge[s->roff[id]];
        if (s->qid[s->qoff[e0] + s->qhead[e0]] == id && !s->is_pending[e0]) {
            s->is_pending[e0] = 1;
            s->pending[s->n_pending++] = e0;
        }
    }

    /* link occupancy sample at the first step of a bin */
    if (p->bin_steps && k % p->bin_steps == 0 && k / p->bin_steps < p->n_bins)
        for (uint32_t a = 0; a < s->n_active_list; a++) {
            uint32_t i = s->active[a];
            s->bin_occ[(uint64_t)s->e[i] * p->n_bins + k / p->bin_steps]++;
        }
    s->veh_steps += s->n_active_list;

    /* P1: every active vehicle, from the state at k */
    for (uint32_t a = 0; a < s->n_active_list; a++) decide(s, s->active[a], k);
    for (uint32_t j = 0; j < s->n_pending; j++) {
        uint32_t e0 = s->pending[j];
        uint32_t h = s->qid[s->qoff[e0] + s->qhead[e0]];
        uint32_t l = entry_lane(s, h, 0);
        s->dreq[j] = (uint8_t)(l == EMPTY ? EMPTY : l);
    }
    /* conflicts on (edge, lane): lowest id wins */
    for (uint32_t a = 0; a < s->n_active_list; a++) {
        uint32_t i = s->active[a];
        if (s->act[i] != ACT_CROSS) continue;
        uint32_t en = s->redge[s->roff[i] + s->r[i] + 1];
        uint64_t slot = s->slot_off[en] + s->tlane[i];
        if (i < s->claim[slot]) s->claim[slot] = i;
    }
    for (uint32_t j = 0; j < s->n_pending; j++) {
        if (s->dreq[j] == EMPTY) continue;
        uint32_t e0 = s->pending[j];
        uint32_t h = s->qid[s->qoff[e0] + s->qhead[e0]];
        uint64_t slot = s->slot_off[e0] + s->dreq[j];
        if (h < s->claim[slot]) s->claim[slot] = h;
    }

    /* P2: write M_nxt (empty at this point) */
    for (uint32_t a = 0; a < s->n_active_list; a++) {
        uint32_t i = s->active[a];
        uint32_t e = s->e[i];
        float L = (float)s->len[e];
        switch (s->act[i]) {
        case ACT_STAY:
        case ACT_INTEND:
            rc = put(s, cell_index(s, e, s->lane[i], (uint32_t)s->xn[i]), speed_byte(s->vn[i]));
            if (rc) return rc;
            break;
        case ACT_CROSS: {
            uint32_t en = s->redge[s->roff[i] + s->r[i] + 1];
            uint64_t slot = s->slot_off[en] + s->tlane[i];
            if (s->claim[slot] == i) {
                stat_exit(s, e, k, s->t_enter[i]);
                s->e[i] = en;
                s->r[i] += 1;
                s->lane[i] = s->tlane[i];
                s->x[i] = 0.0f;
                s->v[i] = s->vn[i];
                s->t_enter[i] = k + 1;
                rc = put(s, cell_index(s, en, s->lane[i], 0), speed_byte(s->v[i]));
                if (rc) return rc;
                stat_entry(s, en, k);
                break;
            }
        }   /* fall through: lost the conflict, wait at the stop line */
        /* FALLTHROUGH */
        case ACT_HOLD: {
            float lim = L - 1.0f;
            s->x[i] = s->x[i] > lim ? s->x[i] : lim;
            s->v[i] = 0.0f;
            rc = put(s, cell_index(s, e, s->lane[i], (uint32_t)s->x[i]), 0);
            if (rc) return rc;
            s->act[i] = ACT_HOLD;
            break;
        }
        case ACT_ARRIVE:
            stat_exit(s, e, k, s->t_enter[i]);
            s->status[i] = ST_ARRIVED;
            s->arr[i] = k + 1;
            s->n_arrived++;
            break;
        default:
            break;
        }
    }
    uint32_t n_next = 0;
    for (uint32_t j = 0; j < s->n_pending; j++) {
        if (s->dreq[j] == EMPTY) continue;
        uint32_t e0 = s->pending[j];
        uint32_t h = s->qid[s->qoff[e0] + s->qhead[e0]];
        uint64_t slot = s->slot_off[e0] + s->dreq[j];
        if (s->claim[slot] != h) continue;
        s->status[h] = ST_ACTIVE;
        s->e[h] = e0;
        s->r[h] = 0;
        s->lane[h] = s->dreq[j];
        s->x[h] = 0.0f;
        s->v[h] = 0.0f;
        s->t_enter[h] = k + 1;
        s->dep_act[h] = k + 1;
        rc = put(s, cell_index(s, e0, s->lane[h], 0), 0);
        if (rc) return rc;
        stat_entry(s, e0, k);
        s->qhead[e0]++;
        s->next_active[n_next++] = h;
    }

    /* P3: lane-change decisions, all against the same maps */
    for (uint32_t a = 0; a < s->n_active_list; a++) {
        uint32_t i = s->active[a];
        s->accept[i] = (s->act[i] == ACT_INTEND) ? (uint8_t)gap_accept(s, i, k) : 0;
    }

    /* P4: apply lane changes, commit positions, erase step-k cells */
    for (uint32_t a = 0; a < s->n_active_list; a++) {
        uint32_t i = s->active[a];
        if (s->accept[i]) {
            uint32_t e = s->e[i], cn = (uint32_t)s->xn[i];
            s->Mnxt[cell_index(s, e, s->lane[i], cn)] = EMPTY;
            s->lane[i] = (uint8_t)((int)s->lane[i] + s->dir[i]);
            rc = put(s, cell_index(s, e, s->lane[i], cn), speed_byte(s->vn[i]));
            if (rc) return rc;
            s->n_lane_changes++;
        }
        if (s->act[i] == ACT_STAY || s->act[i] == ACT_INTEND) {
            s->x[i] = s->xn[i];
            s->v[i] = s->vn[i];
        }
        s->Mcur[s->old_cell[i]] = EMPTY;
    }
    /* claims back to empty: every claimed slot has a winner, and after P2 the
     * only vehicles still marked CROSS are the winners, already on the edge
     * and lane they claimed */
    for (uint32_t a = 0; a < s->n_active_list; a++) {
        uint32_t i = s->active[a];
        if (s->act[i] == ACT_CROSS) s->claim[s->slot_off[s->e[i]] + s->lane[i]] = NO_CLAIM;
    }
    for (uint32_t j = 0; j < s->n_pending; j++)
        if (s->dreq[j] != EMPTY) s->claim[s->slot_off[s->pending[j]] + s->dreq[j]] = NO_CLAIM;

    /* active set for k+1: survivors, then the vehicles that just departed */
    uint32_t m = 0;
    for (uint32_t a = 0; a < s->n_active_list; a++) {
        uint32_t i = s->active[a];
        if (s->status[i] == ST_ACTIVE) s->next_active[n_next + m++] = i;
        s->act[i] = ACT_NONE;
        s->accept[i] = 0;
    }
    /* departures were written first; rotate so survivors come first (order is immaterial) */
    {
        uint32_t *t = s->active;
        s->active = s->next_active;
        s->next_active = t;
        s->n_active_list = n_next + m;
    }
    /* pending edges for k+1: those whose (new) head has been released */
    uint32_t np = 0;
    for (uint32_t j = 0; j < s->n_pending; j++) {
        uint32_t e0 = s->pending[j];
        uint64_t qh = s->qoff[e0] + s->qhead[e0];
        if (qh < s->qoff[e0 + 1] && s->qid[qh] < s->released) s->pending[np++] = e0;
        else s->is_pending[e0] = 0;
    }
    s->n_pending = np;

    uint8_t *t = s->Mcur;
    s->Mcur = s->Mnxt;
    s->Mnxt = t;
    s->k = k + 1;
    return 0;
}

int orc_step(orc_sim *s, uint32_t n_steps) {
    if (!s) return -1;
    if (!s->loaded) return -4;
    for (uint32_t j = 0; j < n_steps; j++) {
        int rc = step_once(s);
        if (rc) return rc;
    }
    return 0;
}

int orc_run(orc_sim *s, uint32_t max_steps, uint64_t *out6) {
    if (!s || !out6) return -1;
    if (!s->loaded) return -4;
    uint64_t vs0 = s->veh_steps;
    uint32_t j = 0;
    while (j < max_steps && s->n_arrived < s->n) {
        int rc = step_once(s);
        if (rc) return rc;
        j++;
    }
    uint64_t waiting = s->n - s->n_arrived - s->n_active_list;
    out6[0] = j;
    out6[1] = s->veh_steps - vs0;
    out6[2] = s->n_arrived;
    out6[3] = s->n_active_list;
    out6[4] = waiting;
    out6[5] = s->k;
    return 0;
}

/* --------------------------------------------------------------- queries */

int orc_get_state(const orc_sim *s, float *x, float *v, uint32_t *edge, uint8_t *lane, uint32_t *ridx,
                  uint8_t *status) {
    if (!s) return -1;
    if (!s->loaded) return -4;
    for (uint64_t i = 0; i < s->n; i++) {
        int act = s->status[i] == ST_ACTIVE;
        if (x) x[i] = act ? s->x[i] : 0.0f;
        if (v) v[i] = act ? s->v[i] : 0.0f;
        if (edge) edge[i] = act ? s->e[i] : 0xFFFFFFFFu;
        if (lane) lane[i] = act ? s->lane[i] : 0;
        if (ridx) ridx[i] = act ? s->r[i] : 0;
        if (status) status[i] = s->status[i];
    }
    return 0;
}

int orc_get_trips(const orc_sim *s, uint32_t *depart_actual, uint32_t *arrive_step) {
    if (!s) return -1;
    if (!s->loaded) return -4;
    for (uint64_t i = 0; i < s->n; i++) {
        if (depart_actual) depart_actual[i] = s->dep_act[i];
        if (arrive_step) arrive_step[i] = s->arr[i];
    }
    return 0;
}

uint64_t orc_lane_map_size(const orc_sim *s) { return s ? s->mcells : 0; }

int orc_get_lane_map(const orc_sim *s, uint8_t *out) {
    if (!s || !out) return -1;
    memcpy(out, s->Mcur, s->mcells);
    return 0;
}

int orc_link_stats(const orc_sim *s, uint64_t *per_edge3, uint32_t *bin_inflow, uint32_t *bin_tt_sum,
                   uint32_t *bin_tt_cnt, uint32_t *bin_occ) {
    if (!s) return -1;
    uint64_t nb = (uint64_t)s->n_edges * s->p.n_bins;
    if (per_edge3)
        for (uint32_t e = 0; e < s->n_edges; e++) {
            per_edge3[3 * (uint64_t)e + 0] = s->ent[e];
            per_edge3[3 * (uint64_t)e + 1] = s->ext[e];
            per_edge3[3 * (uint64_t)e + 2] = s->tts[e];
        }
    if (bin_inflow) memcpy(bin_inflow, s->bin_in, nb * 4);
    if (bin_tt_sum) memcpy(bin_tt_sum, s->bin_tt, nb * 4);
    if (bin_tt_cnt) memcpy(bin_tt_cnt, s->bin_cnt, nb * 4);
    if (bin_occ) memcpy(bin_occ, s->bin_occ, nb * 4);
    return 0;
}

int orc_counters(const orc_sim *s, uint64_t *out6) {
    if (!s || !out6) return -1;
    out6[0] = s->k;
    out6[1] = s->veh_steps;
    out6[2] = s->n_arrived;
    out6[3] = s->n_active_list;
    out6[4] = s->loaded ? s->n - s->n_arrived - s->n_active_list : 0;
    out6[5] = s->n_lane_changes;
    return 0;
}

void orc_destroy(orc_sim *s) {
    if (!s) return;
    void *ptrs[] = {s->src, s->dst, s->len, s->green, s->n_in, s->n_out, s->n_phase, s->v0, s->lanes, s->arank, s->orank,
                    s->moff, s->slot_off, s->Mcur, s->Mnxt, s->dep, s->roff, s->redge, s->status, s->lane,
                    s->act, s->tlane, s->accept, s->dir, s->e, s->r, s->t_enter, s->dep_act, s->arr, s->x,
                    s->v, s->xn, s->vn, s->old_cell, s->active, s->next_active, s->qoff, s->qhead, s->qid,
                    s->pending, s->is_pending, s->dreq, s->claim, s->ent, s->ext, s->tts, s->bin_in,
                    s->bin_tt, s->bin_cnt, s->bin_occ, s->vt};
    for (size_t j = 0; j < sizeof ptrs / sizeof ptrs[0]; j++) free(ptrs[j]);
    free(s);
}
