// Per-step kernels of the vehicle update (Algorithm 1, Sec. 3.1-3.2).
//
// One step k is two launches:
//   step_p1  every live vehicle: leader search in the step-k lane map,
//            IDM / free-flow speed, move with the no-crash clamp, and the
//            decision at the edge end (arrive, ask to cross, hold at the stop
//            line) or the lane-change intent; writes its step-k+1 cell into
//            the next map when it stays; posts entry claims (atomicMin of the
//            vehicle id on the (edge, lane) slot) with a record of what the
//            resolution needs.  Origin edges post the departure claim of
//            their queue head.
//   step_p2  crossers and departures: the lowest id of each claimed slot
//            enters cell 0; the others stop at the stop line.  Lane-change
//            intenders, in the same launch: gap acceptance against the
//            step-k map and the next map; the accepted move their next-map
//            byte sideways.  A stop-line hold can only land on cell len - 1
//            of its own lane, so an intent aiming at any other cell cannot
//            meet one; an intent aiming at a cell len - 1 reads the crossing
//            request made from that lane (at most one: only the lane's front
//            vehicle can reach the stop line) and its claim, which step_p1
//            settled, and so knows whether a hold will land there.  The same
//            launch closes the step (list counts, slot count, crossing log).
//
// Three lane maps rotate: step k reads map[k%3] and writes map[(k+1)%3];
// map[(k+2)%3] still holds the cells of step k-1, which step_p1 erases (each
// vehicle remembers its previous cell), so no step needs a full clear.  The
// intent marks (one byte per cell, imap[k&1]) let an intender see that a
// cell was reserved by another intender even if that one has already moved
// its byte sideways: the result is the same as judging every intender
// against one snapshot, whatever the order the threads run in.
//
// Latency, not bandwidth, bounds these kernels (a step moves a few MB), so
// each is arranged to need as few dependent memory round trips as possible:
// the parity buffers and maps are chosen from a launch argument, the first
// records of a thread are loaded together with the step number and the list
// lengths, and records that a later phase needs are packed by the phase that
// already holds the values.
//
// Every floating-point expression is written in the same operation order as
// the rules state; the library is compiled with -fmad=false -prec-div=true
// -ftz=false, so each operation is one IEEE binary32 rounding.
#include <algorithm>

#include "lpsim_dev.cuh"

namespace lpsim {

namespace {

__device__ __forceinline__ uint64_t splitmix64_mix(uint64_t z) {
    // SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float unit24(uint64_t h) {
    return (float)(uint32_t)(h >> 40) * (1.0f / 16777216.0f);
}

__device__ __forceinline__ float fmax0(float t) { return t > 0.0f ? t : 0.0f; }

__device__ __forceinline__ uint8_t speed_byte(float v) {
    float t = v < 254.0f ? v : 254.0f;
    return (uint8_t)(uint32_t)t;
}

// 16-bit mask of the occupied bytes of a 16-byte chunk.
__device__ __forceinline__ uint32_t occ_mask16(uint4 q) {
    uint32_t w[4] = {q.x, q.y, q.z, q.w};
    uint32_t m = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        uint32_t b = __vcmpne4(w[j], 0xFFFFFFFFu);  // 0xFF per occupied byte
        uint32_t bits = ((b >> 7) & 1u) | ((b >> 14) & 2u) | ((b >> 21) & 4u) | ((b >> 28) & 8u);
        m |= bits << (4 * j);
    }
    return m;
}

__device__ __forceinline__ uint32_t range_mask16(uint32_t c, uint32_t lo, uint32_t hi) {
    // bits of chunk [c, c+16) that fall in [lo, hi]
    uint32_t a = lo > c ? lo - c : 0u;
    uint32_t b = hi < c + 15u ? hi - c : 15u;
    return ((0xFFFFu << a) & (0xFFFFu >> (15u - b))) & 0xFFFFu;
}

// first occupied cell in [lo, hi] of a 16-byte aligned row, or kNone; the
// first four 16-byte chunks of the window are loaded together, so a window of
// up to 49 cells costs one memory round trip
__device__ __forceinline__ uint32_t first_occupied_wide(const uint8_t *row, uint32_t lo, uint32_t hi) {
    if (lo > hi) return kNone;
    const uint32_t c0 = lo & ~15u;
    uint4 q[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const uint32_t c = c0 + 16u * j;
        q[j] = c <= hi ? *reinterpret_cast<const uint4 *>(row + c) : make_uint4(~0u, ~0u, ~0u, ~0u);
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const uint32_t c = c0 + 16u * j;
        if (c > hi) break;
        const uint32_t mk = occ_mask16(q[j]) & range_mask16(c, lo, hi);
        if (mk) return c + (uint32_t)(__ffs((int)mk) - 1);
    }
    for (uint32_t c = c0 + 64u; c <= hi; c += 16u) {
        const uint32_t mk = occ_mask16(*reinterpret_cast<const uint4 *>(row + c)) & range_mask16(c, lo, hi);
        if (mk) return c + (uint32_t)(__ffs((int)mk) - 1);
    }
    return kNone;
}

// car-following parameters of one vehicle (its type's, or the run's)
struct CarParams {
    float a, s0, T, two_sqrt_ab, vmax;
};

__device__ __forceinline__ float idm_speed(const CarParams &y, float dt, float v, float vf, float s, float v0) {
    float dv = v - vf;
    float z = v * y.T + (v * dv) / y.two_sqrt_ab;
    float s_star = y.s0 + fmax0(z);
    float r = v / v0;
    float q = s_star / s;
    float acc = y.a * ((1.0f - (r * r) * (r * r)) - q * q);
    return fmax0(v + acc * dt);
}

// Write a next-map cell.  With the checking flag the cell is read first and
// a second writer is reported in the error word; without it the store does
// not wait for a load (the rules never give one cell two writers).
__device__ __forceinline__ void put_cell(const Dev &d, uint8_t *map, uint32_t idx, uint8_t val) {
    if (d.check && map[idx] != kEmpty) atomicOr(d.err, kErrCellTaken);
    map[idx] = val;
}

__device__ __forceinline__ void stat_entry(const Dev &d, uint32_t e, uint32_t k) {
    atomicAdd(&d.ent[e], 1ull);
    if (d.m.bin_steps) {
        uint32_t b = (k + 1) / d.m.bin_steps;
        if (b < d.m.n_bins) atomicAdd(&d.bin_in[(size_t)b * d.n_edges + e], 1u);
    }
}

__device__ __forceinline__ void stat_exit(const Dev &d, uint32_t e, uint32_t k, uint32_t tent) {
    uint32_t steps = k + 1 - tent;
    atomicAdd(&d.ext[e], 1ull);
    atomicAdd(&d.tts[e], (unsigned long long)steps);
    if (d.m.bin_steps) {
        uint32_t b = tent / d.m.bin_steps;
        if (b < d.m.n_bins) {
            atomicAdd(&d.bin_tt[(size_t)b * d.n_edges + e], steps);
            atomicAdd(&d.bin_cnt[(size_t)b * d.n_edges + e], 1u);
        }
    }
}

// Programmatic dependent launch: let the next kernel of the step sequence be
// scheduled now (its blocks wait in their own prologue), then wait until the
// previous kernel has completed and its writes are visible.
__device__ __forceinline__ void pdl_prologue() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Position in a per-step list for each calling lane: one atomic per group of
// lanes that arrive together (list order does not matter to any result).
__device__ __forceinline__ uint32_t warp_append(uint32_t *counter) {
    const uint32_t mask = __activemask();
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t leader = (uint32_t)__ffs((int)mask) - 1u;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(counter, (uint32_t)__popc((int)mask));
    base = __shfl_sync(mask, base, (int)leader);
    return base + (uint32_t)__popc((int)(mask & ((1u << lane) - 1u)));
}

// Per-block staging of the per-step lists: step_p1 appends an item to shared
// memory (a shared-memory atomic) and the block moves its items to the
// global list with one global atomic at its end, so no thread's chain waits on
// a global round trip for a list position.  Items beyond the room of the
// stage go to the global list directly.
constexpr uint32_t kStageCross = 128, kStageIntend = 128, kStageDep = 64;

static_assert(sizeof(CrossRec) == 64 && sizeof(IntendRec) == 32 && sizeof(DepRec) == 64 && sizeof(RouteRec) == 8,
              "record sizes");

struct P1Sinks {
    CrossRec *cr;
    IntendRec *ir;
    DepRec *dr;
    uint32_t *n;  // [4]: staged crossing requests, intents, departure requests; stop-line intents
};

template <class T>
__device__ __forceinline__ void stage_put(T *buf, uint32_t room, uint32_t *n, T *glist, uint32_t *gcount,
                                          const T &item) {
    const uint32_t pos = atomicAdd(n, 1u);
    if (pos < room)
        buf[pos] = item;
    else
        glist[warp_append(gcount)] = item;
}


// Keeps the loads above it above a following branch (so the first records of
// a thread are in flight while the list length is still on its way).
__device__ __forceinline__ void loads_issued() { asm volatile("" ::: "memory"); }

template <int BLOCK>
__device__ __forceinline__ void block_add(unsigned long long *dst, uint32_t val, unsigned long long *dst2 = nullptr) {
    __shared__ uint32_t red[BLOCK / 32];
    uint32_t w = __reduce_add_sync(0xFFFFFFFFu, val);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t t = threadIdx.x < BLOCK / 32 ? red[threadIdx.x] : 0u;
        t = __reduce_add_sync(0xFFFFFFFFu, t);
        if (threadIdx.x == 0 && t) {
            atomicAdd(dst, (unsigned long long)t);
            if (dst2) atomicAdd(dst2, (unsigned long long)t);
        }
    }
}

// A statistics counter summed over a full warp, then one atomic per warp:
// per-thread atomics on one address serialise in L2 (one per crossing
// vehicle made step_p2 take 60% longer at the morning peak).
__device__ __forceinline__ void warp_add(unsigned long long *dst, uint32_t val) {
    const uint32_t w = __reduce_add_sync(0xFFFFFFFFu, val);
    if ((threadIdx.x & 31u) == 0 && w) atomicAdd(dst, (unsigned long long)w);
}

// the same in 64 bits (a whole chunk's sums)
__device__ __forceinline__ void warp_add64(unsigned long long *dst, uint32_t val) {
    unsigned long long v = val;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31u) == 0 && v) atomicAdd(dst, v);
}

}  // namespace

// ----------------------------------------------------------------------- P1

// Lane asked for when entering an edge: lanes ordered by distance to the
// target lane tl (kNoLane counts as 0; ties to the lower index); the first
// whose cell 0 is empty in the step-k map.  entry_cells reads the up-to-4
// first cells together (it needs only the edge record, so the reads overlap
// the load of tl); kNone if none is empty.
__device__ __forceinline__ uint32_t entry_cells(const uint8_t *Mc, const EdgeRec &er) {
    const uint32_t nl = er.lanes, stride = row_stride(er.len);
    uint32_t empty = 0;  // bit l: cell 0 of lane l is empty
#pragma unroll
    for (uint32_t l = 0; l < 4; l++)
        if (l < nl && Mc[er.moff + l * stride] == kEmpty) empty |= 1u << l;
    return empty;
}

__device__ __forceinline__ uint32_t pick_entry_lane(uint32_t empty, uint32_t nl, uint32_t tl) {
    if (tl == kNoLane) tl = 0;
    for (uint32_t dd = 0; dd < nl; dd++) {
        if (tl >= dd && ((empty >> (tl - dd)) & 1u)) return tl - dd;
        if (dd > 0 && tl + dd < nl && ((empty >> (tl + dd)) & 1u)) return tl + dd;
    }
    return kNone;
}

// The buffers of step k (parity and map rotation from kph, any number
// congruent to k modulo 6).
struct StepView {
    uint32_t k, par;
    const uint8_t *Mc;
    uint8_t *Mn, *Mo;  // next map; map of step k-1 (erased cell by cell)
    uint8_t *Iw, *Io;  // intent marks of step k; of step k-1 (cleared)
    uint32_t *claim, *claim_old;  // entry claims of step k; those won at step k-1 (reset)
    const float *xc, *vc;
    float *xw, *vw;
    bool sample;  // occupancy sample taken at this step
};

__device__ __forceinline__ StepView step_view(const Dev &d, uint32_t k, uint32_t kph) {
    StepView w;
    const uint32_t par = kph & 1u, r3 = kph % 3u;
    w.k = k;
    w.par = par;
    w.Mc = d.map[r3];
    w.Mn = d.map[r3 == 2u ? 0u : r3 + 1u];
    w.Mo = d.map[r3 == 0u ? 2u : r3 - 1u];
    w.Iw = d.imap[par];
    w.Io = d.imap[par ^ 1u];
    w.claim = d.claim[par];
    w.claim_old = d.claim[par ^ 1u];
    w.xc = d.s.x[par];
    w.vc = d.s.v[par];
    w.xw = d.s.x[par ^ 1u];
    w.vw = d.s.v[par ^ 1u];
    w.sample = d.m.bin_steps && (k % d.m.bin_steps == 0) && (k / d.m.bin_steps < d.m.n_bins);
    return w;
}

// Origin edge j: reset the claim its departure won last step; ask for a
// departure of the queue head once its step has come.
__device__ __forceinline__ void p1_origin(const Dev &d, const StepView &w, const P1Sinks &sk, uint32_t j) {
    const uint32_t k = w.k, par = w.par;
    const uint8_t *Mc = w.Mc;
    uint32_t *claim = w.claim, *claim_old = w.claim_old;
    const uint32_t dp = d.dprev[j];
    const QRec hd = d.org_hd[j];
    if (dp != kNone) {
        claim_old[dp] = kNone;
        d.dprev[j] = kNone;
    }
    if (hd.h != kNone && hd.dep <= k) {
        // only a due head needs its origin's records (most origin edges are
        // idle in most steps)
        const EdgeRec er = d.org_rec[j];
        const uint32_t e0 = d.org_edge[j];
        const uint32_t qoff = d.org_qoff[j], qhead = d.org_head[j], qend = d.org_qend[j];
        const RouteRec rr = d.rrec[hd.r0];
        const uint32_t nxt = hd.r0 + 1 < hd.r1 ? d.route[hd.r0 + 1] : kNone;
        const uint32_t so = d.slot_off[e0];
        const uint8_t vt = d.typed ? d.trip_vt[hd.h] : (uint8_t)0;
        const uint32_t l = pick_entry_lane(entry_cells(Mc, er), er.lanes, rr.tl);
        if (l != kNone) {
            atomicMin(&claim[so + l], hd.h);
            DepRec dr;
            dr.j = j;
            dr.slot = so + l;
            dr.h = hd.h;
            dr.r0 = hd.r0;
            dr.r1 = hd.r1;
            dr.qoff = qoff;
            dr.qhead = qhead;
            dr.qend = qend;
            dr.base = er.moff + l * row_stride(er.len);
            dr.e0 = e0;
            dr.nen = nxt;
            dr.nsg = rr.green;
            dr.v0 = er.v0;
            dr.len = er.len;
            dr.nsph = (uint16_t)(rr.nphase | (rr.arank << 8));
            dr.lane = (uint8_t)l;
            dr.tlc = rr.tl;
            dr.vt = vt;
            stage_put(sk.dr, kStageDep, sk.n + 2, d.dep_rec[par], &d.counts[4 + par], dr);
        }
    }
}

// Slot s (every field loaded in one round trip, together with whatever the
// caller loaded just before); false once s is past the slot count n.
__device__ __forceinline__ bool p1_slot(const Dev &d, const StepView &w, const P1Sinks &sk, uint32_t s, uint32_t n,
                                        uint32_t &live, uint32_t &arrived) {
    const uint32_t k = w.k, par = w.par;
    const uint8_t *Mc = w.Mc;
    uint8_t *Mn = w.Mn, *Mo = w.Mo, *Iw = w.Iw, *Io = w.Io;
    uint32_t *claim = w.claim, *claim_old = w.claim_old;
    const float *xc = w.xc, *vc = w.vc;
    float *xw = w.xw, *vw = w.vw;
    const bool sample = w.sample;
    const Model &m = d.m;
    // every slot field, loaded together (one memory round trip, shared
    // with the loads of the step number and the slot count)
    const uint8_t flag = d.s.flag[s];
    const uint32_t pc = d.s.pcell[s];
    const uint32_t im = d.s.imark[s];
    const uint32_t cp = d.s.cprev[s];
    const float x = xc[s], v = vc[s];
    const EdgeState es = load_es(d.s.es + s);
    const uint32_t base = es.base;
    const uint32_t len = es.len;
    const uint32_t en = es.en;
    const uint32_t G = es.sg;
    const uint32_t ph = es.sph;
    const uint32_t tl = d.s.tlc[s];  // kNoLane on the last edge of the route
    const uint32_t ln = d.s.lane[s];
    const uint32_t id = d.s.id[s];
    const uint32_t rpos = es.rpos, rlast = d.s.rlast[s];
    loads_issued();
    if (s >= n) return false;
    if (flag == kDead) return true;
    if (pc != kNone) Mo[pc] = kEmpty;
    if (im != kNone) {
        Io[im] = 0;
        d.s.imark[s] = kNone;
    }
    if (cp != kNone) {
        claim_old[cp] = kNone;
        d.s.cprev[s] = kNone;
    }
    if (flag == kArrivedPending) {
        d.s.flag[s] = kDead;
        d.s.pcell[s] = kNone;
        return true;
    }
    live++;
    const uint32_t c = (uint32_t)x;
    d.s.pcell[s] = base + c;
    if (sample) atomicAdd(&d.bin_occ[(size_t)(k / m.bin_steps) * d.n_edges + d.route[rpos]], 1u);

    // the vehicle's car-following parameters: its type's (recorded in the
    // edge-state record), or the run's; its free-flow speed is the lower of
    // the edge limit and its top speed
    CarParams y{m.a, m.s0, m.T, m.two_sqrt_ab, 254.0f};
    if (d.typed) {
        const TypeRec tr = d.types[es.vt];
        y = CarParams{tr.a, tr.s0, tr.T, tr.two_sqrt_ab, tr.vmax};
    }
    const float v0 = es.v0 < y.vmax ? es.v0 : y.vmax;
    // leader: nearest occupied cell ahead in the own lane of the own edge.
    // Cells beyond both d_front and the farthest reach of this step
    // cannot change the result, so the scan stops there.
    const float d_front = (2.0f * m.dt) * v;
    const float vmax_step = fmaxf(v0, v + y.a * m.dt);
    const float reach = fmaxf(d_front, vmax_step * m.dt + y.s0);
    const float L = (float)len;
    // in the same round trip as the scan: the next edge's records for a
    // vehicle that may reach the stop line, the lane-change key for one
    // that may draw (both only used under the exact conditions below)
    const bool may_end = x + vmax_step * m.dt + 1.0f >= L;  // may reach the stop line (or arrive)
    // the signal of the edge end, from the slot record: a vehicle facing red
    // only holds, so it needs none of the crossing records
    const bool green = may_end && en != kNone && (G == 0 || (k / G) % (ph & 0xFFu) == (ph >> 8));
    const bool may_cross = green;
    const bool may_draw = tl != kNoLane && tl != ln && ((tl > ln) == (par == 1u)) && (L - x) < m.x0;
    float nv0 = 0.0f;
    RouteRec rr{};
    uint32_t nen = kNone, e = kNone, tent = 0, empty = 0, so = 0;
    if (may_cross || (may_end && en == kNone)) {
        // the current edge and its entry step (for the statistics of a
        // crossing or an arrival)
        e = d.route[rpos];
        tent = d.s.tent[s];
    }
    if (may_cross) {
        nv0 = d.edge[en].v0;
        rr = d.rrec[rpos + 1];
        nen = rpos + 1 < rlast ? d.route[rpos + 2] : kNone;
        so = d.slot_off[en];
        // entry cells of the next edge, from the geometry kept in the slot
        const uint32_t stride = row_stride(es.nlen);
#pragma unroll
        for (uint32_t l = 0; l < 4; l++)
            if (l < es.nlanes && Mc[es.nmoff + l * stride] == kEmpty) empty |= 1u << l;
    }
    // lane-change draw at step k: SplitMix64 of hkey ^ k * C2, where
    // hkey[id] = seed ^ local_id * C1 was formed at load time (local_id =
    // the vehicle's id within its scenario, so a scenario draws the same
    // numbers alone or inside a batch)
    const uint64_t hk = !may_draw ? 0ull
                        : d.hkey_from_id ? d.m.seed ^ ((uint64_t)id * 0x9E3779B97F4A7C15ull)
                                         : d.hkey[id];
    uint32_t hi = c + (uint32_t)fminf(reach, 65535.0f) + 2u;
    if (hi > len - 1) hi = len - 1;
    const uint32_t cf = first_occupied_wide(Mc + base, c + 1, hi);
    const bool has_f = cf != kNone;

    float vn;
    if (has_f && ((float)cf - x) <= d_front)
        vn = idm_speed(y, m.dt, v, (float)Mc[base + cf], (float)cf - x, v0);
    else
        vn = v0;
    float xn = x + vn * m.dt;
    if (has_f) {
        const float lim = (float)cf - y.s0;
        if (xn > lim) {
            xn = x > lim ? x : lim;
            vn = 0.0f;
        }
    }
    if (xn >= L) {
        if (en == kNone) {
            // last edge of the route: arrive (may_end holds: x' <= x + vmax_step * dt)
            stat_exit(d, e, k, tent);
            d.arr[id] = k + 1;
            d.status[id] = kArrived;
            d.s.flag[s] = kArrivedPending;
            arrived++;
            return true;
        }
        bool cross = false;
        if (green) {
            // may_cross holds here: x' >= L needs x + vmax_step * dt >= L
            const uint32_t l = pick_entry_lane(empty, es.nlanes, rr.tl);
            if (l != kNone) {
                const uint32_t slot = so + l;
                atomicMin(&claim[slot], id);
                d.xreq[base >> 4] = make_uint4(k, slot, id, 0u);
                CrossRec cr;
                cr.s = s;
                cr.id = id;
                cr.cslot = slot;
                cr.e = e;
                cr.en = en;
                cr.rpos = rpos;
                cr.tent = tent;
                cr.base = base;
                cr.nbase = es.nmoff + l * row_stride(es.nlen);
                cr.nen = nen;
                cr.nsg = rr.green;
                cr.x = x;
                cr.vn = vn;
                cr.nv0 = nv0;
                cr.len = (uint16_t)len;
                cr.nlen = es.nlen;
                cr.nsph = (uint16_t)(rr.nphase | (rr.arank << 8));
                cr.lane = (uint8_t)(l | ((uint32_t)es.vt << 2));  // lane 0..3, the type above it
                cr.tln = rr.tl;
                stage_put(sk.cr, kStageCross, sk.n, d.cross_list[par], &d.counts[par], cr);
                cross = true;
            }
        }
        if (!cross) {
            const float lim = L - 1.0f;
            const float xh = x > lim ? x : lim;
            xw[s] = xh;
            vw[s] = 0.0f;
            put_cell(d, Mn, base + (uint32_t)xh, 0);
        }
        return true;
    }
    xw[s] = xn;
    vw[s] = vn;
    const uint32_t cn = (uint32_t)xn;
    put_cell(d, Mn, base + cn, speed_byte(vn));
    bool intend = false;
    uint32_t up = 0;
    uint64_t hkd = hk;
    if (may_draw) {
        const float xrem = L - x;
        const float mp = xrem >= m.x0 ? 0.0f : 1.0f - xrem / m.x0;
        // u is in [0, 1): no draw can pass when mp <= 0
        if (mp > 0.0f && unit24(splitmix64_mix(hk ^ ((uint64_t)k * 0xD1B54A32D192ED03ull))) < mp) {
            intend = true;
            up = tl > ln ? 1u : 0u;
        }
    } else if (m.dlc_prob > 0.0f && has_f && vn < v0 && !(tl != kNoLane && tl != ln && (L - x) < m.x0) &&
               (float)Mc[base + cf] < v0) {
        // discretionary lane change (outside the mandatory zone, held below
        // its free speed by a slower leader): one lane up on odd steps, down
        // on even ones, when that lane's lead gap is absent or longer by
        // dlc_gain; the same draw as the mandatory rule
        up = par;
        const uint32_t nl = d.edge[d.route[rpos]].lanes;
        if (up ? ln + 1 < nl : ln > 0) {
            const uint32_t stride = row_stride(len);
            const uint32_t base2 = up ? base + stride : base - stride;
            const uint32_t ca = first_occupied_wide(Mc + base2, c, min(c + 63u, len - 1));
            if (ca == kNone || (float)ca - (float)cf >= m.dlc_gain) {
                hkd = d.hkey_from_id ? d.m.seed ^ ((uint64_t)id * 0x9E3779B97F4A7C15ull) : d.hkey[id];
                intend = unit24(splitmix64_mix(hkd ^ ((uint64_t)k * 0xD1B54A32D192ED03ull))) < m.dlc_prob;
            }
        }
    }
    if (intend) {
        Iw[base + cn] = 1;
        d.s.imark[s] = base + cn;
        IntendRec ir;
        ir.s = s;
        ir.base = base;
        ir.hk = hkd;
        ir.x = x;
        ir.xn = xn;
        ir.vn = vn;
        ir.len = (uint16_t)len;
        ir.lane = (uint8_t)ln;
        ir.up = (uint8_t)up;
        // An intent aiming at cell len - 1 (where a stop-line hold may land) goes to
        // the top of the same list, growing downwards: step_p2 checks those few
        // against the crossing request of the target lane.
        if (cn + 1 < len)
            stage_put(sk.ir, kStageIntend, sk.n + 1, d.intend_list[par], &d.counts[2 + par], ir);
        else {
            d.intend_list[par][d.cap - 1 - warp_append(&d.counts[6 + par])] = ir;
            atomicAdd(sk.n + 3, 1u);
        }
    }
    return true;
}

// 16-byte words of the staged records into a global list (every thread)
template <class T>
__device__ __forceinline__ void stage_copy(const T *buf, uint32_t cnt, T *glist, uint32_t base) {
    const uint32_t words = cnt * (uint32_t)(sizeof(T) / 16);
    const uint4 *src = reinterpret_cast<const uint4 *>(buf);
    uint4 *dst = reinterpret_cast<uint4 *>(glist + base);
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
}

// The block's staged records to the step's lists (after a block barrier):
// the three list positions are reserved by three threads at once (one
// global round trip), then every thread copies.
__device__ __forceinline__ void p1_flush(const Dev &d, uint32_t par, const P1Sinks &sk, uint32_t *s_base) {
    if (threadIdx.x < 3) {
        const uint32_t room = threadIdx.x == 0 ? kStageCross : threadIdx.x == 1 ? kStageIntend : kStageDep;
        const uint32_t cnt = min(sk.n[threadIdx.x], room);
        s_base[threadIdx.x] = cnt ? atomicAdd(&d.counts[2 * threadIdx.x + par], cnt) : 0u;
    }
    __syncthreads();
    stage_copy(sk.cr, min(sk.n[0], kStageCross), d.cross_list[par], s_base[0]);
    stage_copy(sk.ir, min(sk.n[1], kStageIntend), d.intend_list[par], s_base[1]);
    stage_copy(sk.dr, min(sk.n[2], kStageDep), d.dep_rec[par], s_base[2]);
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) step_p1(Dev d, uint32_t koff, uint32_t kph) {
    pdl_prologue();
    span_start(d, 3 * koff);
    const uint32_t k = *d.kbase + koff;
    const uint32_t n = *d.n_slots;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        d.snap[0] = n;
        d.snap[1] = *d.ev_n;
    }
    const StepView w = step_view(d, k, kph);
    const uint32_t norg = d.n_org;
    const uint32_t lim = norg + d.cap;  // items: origin edges first, then slots
    __shared__ __align__(16) CrossRec s_cr[kStageCross];
    __shared__ __align__(16) IntendRec s_ir[kStageIntend];
    __shared__ __align__(16) DepRec s_dr[kStageDep];
    __shared__ uint32_t s_n[4], s_base[3];
    if (threadIdx.x < 4) s_n[threadIdx.x] = 0;
    __syncthreads();
    const P1Sinks sk{s_cr, s_ir, s_dr, s_n};
    uint32_t live = 0;
    uint32_t arrived = 0;
    for (uint32_t i = blockIdx.x * BLOCK + threadIdx.x; i < lim; i += gridDim.x * BLOCK) {
        if (i < norg) {
            p1_origin(d, w, sk, i);
            continue;
        }
        if (!p1_slot(d, w, sk, i - norg, n, live, arrived)) break;
    }
    block_add<BLOCK>(&d.ctr[0], live, d.tacc ? &d.tacc[8] : nullptr);
    warp_add(&d.ctr[1], arrived);
    p1_flush(d, w.par, sk, s_base);
    span_end(d, 3 * koff);
}

// ----------------------------------------------------------------------- P2

// Crossing request cr: the lowest id asking for the (edge, lane) enters its
// cell 0, the others hold at the stop line.
__device__ __forceinline__ void p2_cross(const Dev &d, const StepView &w, const CrossRec &cr, uint32_t ev,
                                         uint32_t &events) {
    const uint32_t k = w.k;
    uint8_t *Mn = w.Mn;
    float *xw = w.xw, *vw = w.vw;
    // the edge after the next one (for the record of a winner), loaded with the claim
    const EdgeRec nn = cr.nen != kNone ? d.edge[cr.nen] : EdgeRec{0, 0, 0, 0, 0.0f, 0};
    if (w.claim[cr.cslot] == cr.id) {
        const uint32_t s = cr.s;
        if (ev < d.ev_cap) {
            d.ev_log[ev] = make_uint4(cr.e, cr.en, cr.tent, k);
        } else {
            stat_exit(d, cr.e, k, cr.tent);
            stat_entry(d, cr.en, k);
        }
        EdgeState ne;
        ne.base = cr.nbase;
        ne.rpos = cr.rpos + 1;
        ne.en = cr.nen;
        ne.sg = cr.nsg;
        ne.v0 = cr.nv0;
        ne.nmoff = nn.moff;
        ne.len = cr.nlen;
        ne.sph = cr.nsph;
        ne.nlen = nn.len;
        ne.nlanes = nn.lanes;
        ne.vt = (uint8_t)(cr.lane >> 2);
        store_es(d.s.es + s, ne);
        d.s.tent[s] = k + 1;
        d.s.lane[s] = (uint8_t)(cr.lane & 3u);
        d.s.tlc[s] = cr.tln;
        d.s.cprev[s] = cr.cslot;
        xw[s] = 0.0f;
        vw[s] = cr.vn;
        put_cell(d, Mn, cr.nbase, speed_byte(cr.vn));
        events++;
    } else {
        if (ev < d.ev_cap) d.ev_log[ev] = make_uint4(kNone, 0u, 0u, 0u);
        const float lim = (float)cr.len - 1.0f;
        const float xh = cr.x > lim ? cr.x : lim;
        xw[cr.s] = xh;
        vw[cr.s] = 0.0f;
        put_cell(d, Mn, cr.base + (uint32_t)xh, 0);
    }
}

// Departure request number q (slot n0 + q, fixed in advance): the queue head
// enters cell 0 of its first edge if it holds the lowest id asking for it.
__device__ __forceinline__ void p2_dep(const Dev &d, const StepView &w, const DepRec &dr, uint32_t q, uint32_t n0,
                                       uint32_t &events, uint32_t &departed) {
    const uint32_t k = w.k;
    const uint32_t s = n0 + q;
    const uint32_t qh = dr.qoff + dr.qhead;
    const QRec next = qh + 1 < dr.qend ? d.qrec[qh + 1] : QRec{kNone, kNone, 0, 0};
    const uint32_t won = w.claim[dr.slot];
    const EdgeRec nn = dr.nen != kNone ? d.edge[dr.nen] : EdgeRec{0, 0, 0, 0, 0.0f, 0};
    if (s >= d.cap) {
        atomicOr(d.err, kErrSlotOverflow);
        return;
    }
    if (won != dr.h) {
        d.s.flag[s] = kDead;
        d.s.pcell[s] = kNone;
        d.s.imark[s] = kNone;
        d.s.cprev[s] = kNone;
        return;
    }
    EdgeState ne;
    ne.base = dr.base;
    ne.rpos = dr.r0;
    ne.en = dr.nen;
    ne.sg = dr.nsg;
    ne.v0 = dr.v0;
    ne.nmoff = nn.moff;
    ne.len = dr.len;
    ne.sph = dr.nsph;
    ne.nlen = nn.len;
    ne.nlanes = nn.lanes;
    ne.vt = dr.vt;
    store_es(d.s.es + s, ne);
    d.s.tent[s] = k + 1;
    d.s.id[s] = dr.h;
    d.s.rlast[s] = dr.r1 - 1;
    d.s.lane[s] = dr.lane;
    d.s.tlc[s] = dr.tlc;
    d.s.pcell[s] = kNone;
    d.s.imark[s] = kNone;
    d.s.cprev[s] = kNone;
    d.s.flag[s] = kLive;
    w.xw[s] = 0.0f;
    w.vw[s] = 0.0f;
    put_cell(d, w.Mn, dr.base, 0);
    d.dprev[dr.j] = dr.slot;
    d.org_head[dr.j] = dr.qhead + 1;
    d.org_hd[dr.j] = next;
    d.dep_act[dr.h] = k + 1;
    d.status[dr.h] = kActive;
    stat_entry(d, dr.e0, k);
    events++;
    departed++;
}

// ----------------------------------------------------------------------- P3

// occupancy masks of the 5 chunks covering [c0 - 64, c0 + 63] around an
// aligned base (loaded together)
template <int N>
__device__ __forceinline__ void load_chunks(const uint8_t *row, uint32_t c_first, uint32_t c_last, uint32_t (&mk)[N]) {
    uint4 q[N];
#pragma unroll
    for (int j = 0; j < N; j++) {
        const uint32_t c = c_first + 16u * j;
        q[j] = c <= c_last ? *reinterpret_cast<const uint4 *>(row + c) : make_uint4(~0u, ~0u, ~0u, ~0u);
    }
#pragma unroll
    for (int j = 0; j < N; j++) mk[j] = occ_mask16(q[j]);
}

// Lane-change intender ir: gap acceptance against the step-k map and the
// reservations of the next map; the accepted move their byte sideways.  With
// `late` (the intent aims at cell len - 1 and runs alongside the crossing
// requests) a hold that a losing crosser of the target lane is placing in the
// same kernel counts as occupying the target cell.
__device__ __forceinline__ void lane_change(const Dev &d, const StepView &w, const IntendRec &ir, uint32_t &changes,
                                          bool late) {
    const uint32_t k = w.k;
    const uint8_t *Mc = w.Mc;
    uint8_t *Mn = w.Mn;
    const uint8_t *Iw = w.Iw;
    const Model &m = d.m;
    const uint32_t s = ir.s;
    const uint32_t ln = ir.lane;
    const bool up = ir.up != 0;
    const uint32_t len = ir.len, stride = row_stride(len);
    const uint32_t base = ir.base;
    const float x = ir.x, xn = ir.xn, vn = ir.vn;
    const uint32_t base2 = up ? base + stride : base - stride;
    const uint8_t *row2 = Mc + base2;
    const uint32_t c0 = (uint32_t)x, cn = (uint32_t)xn;
    // window [c0 - 64, c0 + 63] of the target lane, clipped to the row
    const uint32_t lo = c0 > 64u ? c0 - 64u : 0u;
    const uint32_t hi = c0 + 63u < len - 1 ? c0 + 63u : len - 1;
    const uint32_t cfirst = lo & ~15u;
    uint32_t mk[9];
    load_chunks<9>(row2, cfirst, hi, mk);
    const uint32_t tgt = base2 + cn;
    const uint8_t tgt_map = Mn[tgt], tgt_mark = Iw[tgt];
    const uint4 xr = late ? d.xreq[base2 >> 4] : make_uint4(kNone, 0u, 0u, 0u);
    uint64_t h = 0;
    if (m.eps_amp > 0.0f) h = splitmix64_mix(ir.hk ^ ((uint64_t)k * 0xD1B54A32D192ED03ull));
    // lead: first occupied cell in [c0, hi]; lag: last in [lo, c0 - 1]
    uint32_t ca = kNone, cb = kNone;
#pragma unroll
    for (int j = 0; j < 9; j++) {
        const uint32_t c = cfirst + 16u * j;
        if (c > hi) break;
        const uint32_t a = mk[j] & range_mask16(c, c0, hi);
        if (ca == kNone && a) ca = c + (uint32_t)(__ffs((int)a) - 1);
        if (c0 > 0 && c <= c0 - 1) {
            const uint32_t b = mk[j] & range_mask16(c, lo, c0 - 1);
            if (b) cb = c + (31u - (uint32_t)__clz((int)b));
        }
    }
    float eps_a = 0.0f, eps_b = 0.0f;
    if (m.eps_amp > 0.0f) {
        eps_a = m.eps_amp * (2.0f * unit24(splitmix64_mix(h ^ 0x632BE59BD9B4E019ull)) - 1.0f);
        eps_b = m.eps_amp * (2.0f * unit24(splitmix64_mix(h ^ 0x8CB92BA72F3D8DD7ull)) - 1.0f);
    }
    bool ok = true;
    if (ca != kNone) {
        const float va = (float)row2[ca];
        const float G_lead = (m.g_a + fmax0(m.alpha_i * vn - m.alpha_a * va)) + eps_a;
        ok = ((float)ca - xn) >= G_lead;
    }
    if (ok && cb != kNone) {
        const float vb = (float)row2[cb];
        const float G_lag = (m.g_b + fmax0(m.alpha_b * vb - m.alpha_i * vn)) + eps_b;
        ok = (xn - (float)cb) >= G_lag;
    }
    // a crossing request from the target lane at this step that lost its
    // claim holds at cell len - 1, the target cell of a late intent
    if (ok && xr.x == k) ok = w.claim[xr.y] == xr.z;
    if (ok && cn >= 1 && tgt_map == kEmpty && tgt_mark == 0) {
        // the own next cell holds the byte step P1 wrote there (its intent
        // mark keeps every other mover out of it)
        Mn[tgt] = speed_byte(vn);
        Mn[base + cn] = kEmpty;
        d.s.lane[s] = (uint8_t)(up ? ln + 1 : ln - 1);
        d.s.es[s].base = base2;
        changes++;
    }
}

// Blocks [0, gc) take the crossing requests, [gc, gc + gi) the lane-change
// intents aiming at a cell no stop-line hold can take, block gc + gi those
// aiming at a cell len - 1, the last gdep (enough for one request per origin
// edge) the departure requests; each thread's first record is loaded
// together with its list's length.  Thread 0 of block 0 closes the step: the
// next step's lists start empty, this step's departures have taken their
// slots and its crossings their log entries (every other thread reads the
// step's starting values from the snapshot step_p1 took).
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) step_p2(Dev d, uint32_t koff, uint32_t kph, uint32_t gc, uint32_t gi) {
    pdl_prologue();
    span_start(d, 3 * koff + 1);
    const uint32_t par = kph & 1u;
    const uint32_t k = *d.kbase + koff;
    const StepView w = step_view(d, k, kph);
    const bool closer = blockIdx.x == 0 && threadIdx.x == 0;
    uint32_t ndep_c = 0, ns = 0;
    if (closer) {
        ndep_c = d.counts[4 + par];
        ns = d.snap[0];
    }
    uint32_t events = 0, departed = 0, changes = 0;
    if (blockIdx.x < gc) {
        const uint32_t ncross = d.counts[par];
        const uint32_t ev0 = d.snap[1];  // this step's crossings follow the chunk's earlier ones in the log
        const CrossRec *list = d.cross_list[par];
        // item i goes to block i % gc: a short list spreads over every block (and SM)
        for (uint32_t i = threadIdx.x * gc + blockIdx.x; i < d.cap; i += gc * BLOCK) {
            const CrossRec cr = list[i];
            loads_issued();
            if (i >= ncross) break;
            p2_cross(d, w, cr, ev0 + i, events);
        }
        if (closer) {
            d.counts[par ^ 1u] = 0;
            d.counts[2 + (par ^ 1u)] = 0;
            d.counts[4 + (par ^ 1u)] = 0;
            d.counts[6 + (par ^ 1u)] = 0;
            *d.n_slots = ns + ndep_c;
            *d.ev_n = ev0 + ncross;
        }
    } else if (blockIdx.x < gc + gi) {
        const uint32_t nint = d.counts[2 + par];
        const IntendRec *list = d.intend_list[par];
        for (uint32_t i = threadIdx.x * gi + (blockIdx.x - gc); i < d.cap; i += gi * BLOCK) {
            const IntendRec ir = list[i];
            loads_issued();
            if (i >= nint) break;
            lane_change(d, w, ir, changes, false);
        }
    } else if (blockIdx.x == gc + gi) {
        const uint32_t nlate = d.counts[6 + par];
        const IntendRec *top = d.intend_list[par] + (d.cap - 1);
        for (uint32_t i = threadIdx.x; i < d.cap; i += BLOCK) {
            const IntendRec ir = *(top - i);
            loads_issued();
            if (i >= nlate) break;
            lane_change(d, w, ir, changes, true);
        }
    } else {
        const uint32_t ndep = d.counts[4 + par];
        const uint32_t n0 = d.snap[0];
        const uint32_t b0 = gc + gi + 1;
        const uint32_t nthr = (gridDim.x - b0) * BLOCK;
        const DepRec *list = d.dep_rec[par];
        for (uint32_t q = (blockIdx.x - b0) * BLOCK + threadIdx.x; q < d.n_org; q += nthr) {
            const DepRec dr = list[q];
            loads_issued();
            if (q >= ndep) break;
            p2_dep(d, w, dr, q, n0, events, departed);
        }
    }
    warp_add(&d.ctr[3], events);
    warp_add(&d.ctr[4], departed);
    warp_add(&d.ctr[2], changes);
    span_end(d, 3 * koff + 1);
}

// ------------------------------------------------------------ light load

// Many steps in one block when few vehicles move: the three phases of a
// step are separated by block barriers instead of kernel boundaries.  The
// host picks this kernel for a chunk only when few trips can be on the
// network or waiting during it; olist holds the origin edges that can act in
// the chunk (a queue head due before its end, or a claim to reset).  Every
// phase body is the one the grid-wide kernels run, so the results are the
// same.  What the grid-wide kernels pass through global memory stays on chip
// here: the per-step lists are read from the block's stages (only items
// beyond a stage's room go through the global lists, from position 0), the
// list lengths come from the stage counters, the slot count and the crossing
// log position live in registers and the statistics counters are summed
// over the whole chunk.  A step then costs three block barriers and no
// global round trip of its own.  (Clusters of 2-8 such blocks, synchronised
// by cluster barriers, were measured slower than the grid-wide kernels for
// 2k-12k trips.)
// map_words > 0: the network's five lane maps (three rotating occupancy
// maps, two intent maps; map_words 16-byte words each) are copied into this
// block's shared memory for the chunk and back at its end, and every phase
// reads and writes them there (through generic addresses: the phase bodies
// are the same code); 0: they stay in global memory.
__global__ void __launch_bounds__(kSmallBlock, 1)
    step_small(Dev d, uint32_t k0, uint32_t nsteps, const uint32_t *olist, const uint32_t *no_ptr,
               uint32_t map_words) {
    extern __shared__ __align__(16) uint4 s_maps[];
    span_start(d, d.tspan_light);
    const uint32_t tid = threadIdx.x;
    const uint32_t no = *no_ptr;
    uint32_t n = *d.n_slots, ev0 = *d.ev_n;
    // the five maps in global memory, in the order (map 0, 1, 2, intent map 0, 1)
    uint8_t *const gmaps[5] = {d.map[0], d.map[1], d.map[2], d.imap[0], d.imap[1]};
    if (map_words) {
        for (int a = 0; a < 5; a++) {
            const uint4 *g = reinterpret_cast<const uint4 *>(gmaps[a]);
            uint4 *sm = s_maps + (size_t)a * map_words;
            for (uint32_t i = tid; i < map_words; i += kSmallBlock) sm[i] = g[i];
        }
    }
    __shared__ __align__(16) CrossRec s_cr[kStageCross];
    __shared__ __align__(16) IntendRec s_ir[kStageIntend];
    __shared__ __align__(16) DepRec s_dr[kStageDep];
    __shared__ uint32_t s_n[4];
    const P1Sinks sk{s_cr, s_ir, s_dr, s_n};
    if (tid < 4) s_n[tid] = 0;
    __syncthreads();
    uint32_t live = 0, arrived = 0, events = 0, departed = 0, changes = 0;
    for (uint32_t t = 0; t < nsteps; t++) {
        const uint32_t k = k0 + t, par = k & 1u;
        StepView w = step_view(d, k, k);
        if (map_words) {
            // the same rotation over the shared-memory copies
            uint8_t *const sm = reinterpret_cast<uint8_t *>(s_maps);
            const size_t mb = (size_t)map_words * 16;
            const uint32_t r3 = k % 3u;
            w.Mc = sm + r3 * mb;
            w.Mn = sm + (r3 == 2u ? 0u : r3 + 1u) * mb;
            w.Mo = sm + (r3 == 0u ? 2u : r3 - 1u) * mb;
            w.Iw = sm + (3u + par) * mb;
            w.Io = sm + (3u + (par ^ 1u)) * mb;
        }
        // P1
        for (uint32_t i = tid; i < no; i += kSmallBlock) p1_origin(d, w, sk, olist[i]);
        for (uint32_t s = tid; s < n; s += kSmallBlock) p1_slot(d, w, sk, s, n, live, arrived);
        __syncthreads();
        // P2: staged items first, then the overflow in the global lists
        const uint32_t ncross = s_n[0], nint = s_n[1], ndep = s_n[2], nlate = s_n[3];
        for (uint32_t i = tid; i < ncross; i += kSmallBlock)
            p2_cross(d, w, i < kStageCross ? s_cr[i] : d.cross_list[par][i - kStageCross], ev0 + i, events);
        for (uint32_t i = tid; i < nint; i += kSmallBlock)
            lane_change(d, w, i < kStageIntend ? s_ir[i] : d.intend_list[par][i - kStageIntend], changes, false);
        for (uint32_t q = tid; q < ndep; q += kSmallBlock)
            p2_dep(d, w, q < kStageDep ? s_dr[q] : d.dep_rec[par][q - kStageDep], q, n, events, departed);
        __syncthreads();
        // P3 (every thread has read the stage counters: the next step's start here)
        if (tid < 4) s_n[tid] = 0;
        for (uint32_t i = tid; i < nlate; i += kSmallBlock)
            lane_change(d, w, d.intend_list[par][d.cap - 1 - i], changes, false);
        if (tid == 0) {  // the next step's global lists start empty
            d.counts[par ^ 1u] = 0;
            d.counts[2 + (par ^ 1u)] = 0;
            d.counts[4 + (par ^ 1u)] = 0;
            d.counts[6 + (par ^ 1u)] = 0;
        }
        n += ndep;
        ev0 += ncross;
        __syncthreads();
    }
    if (tid == 0) {
        *d.n_slots = n;
        *d.ev_n = ev0;
    }
    if (map_words) {
        // the loop ended on a block barrier: every write to the maps is done
        for (int a = 0; a < 5; a++) {
            const uint4 *sm = s_maps + (size_t)a * map_words;
            uint4 *g = reinterpret_cast<uint4 *>(gmaps[a]);
            for (uint32_t i = tid; i < map_words; i += kSmallBlock) g[i] = sm[i];
        }
    }
    warp_add64(&d.ctr[0], live);
    warp_add64(&d.ctr[1], arrived);
    warp_add64(&d.ctr[2], changes);
    warp_add64(&d.ctr[3], events);
    warp_add64(&d.ctr[4], departed);
    span_end(d, d.tspan_light);
}

// Origin edges that can act in steps [k0, k1): a queue head due before k1,
// or a claim won at the previous step still to reset.
__global__ void small_origins(Dev d, uint32_t k1, uint32_t *olist, uint32_t *no) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < d.n_org; j += gridDim.x * blockDim.x) {
        const QRec hd = d.org_hd[j];
        if (d.dprev[j] != kNone || (hd.h != kNone && hd.dep < k1)) olist[warp_append(no)] = j;
    }
}

// per trip: the route records of its positions
__global__ void route_records(Dev d, uint64_t n, RouteRec *out) {
    for (uint64_t h = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; h < n; h += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r0 = d.roff[h], r1 = d.roff[h + 1];
        for (uint32_t q = r0; q < r1; q++) {
            const EdgeRec er = d.edge[d.route[q]];
            const NodeRec nr = d.node[er.dst];
            RouteRec rr;
            rr.green = nr.green;
            rr.nphase = nr.nphase;
            rr.arank = er.arank;
            rr.tl = q + 1 < r1 ? (uint8_t)(((uint32_t)d.orank[d.route[q + 1]] * er.lanes) / nr.nout) : kNoLane;
            rr.pad = 0;
            out[q] = rr;
        }
    }
}

// the crossing log of the chunk into the link statistics
__global__ void apply_crossings(Dev d) {
    const uint32_t n = min(*d.ev_n, d.ev_cap);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint4 r = d.ev_log[i];
        if (r.x == kNone) continue;
        stat_exit(d, r.x, r.w, r.z);
        stat_entry(d, r.y, r.w);
    }
}

// kernel timing: fold the spans of steps [0, nsteps) of the chunk and of the
// light-load kernel into the accumulators and clear their slots (one block)
__global__ void __launch_bounds__(1024) timing_fold(Dev d, uint32_t nsteps) {
    __shared__ unsigned long long red[8][32];
    unsigned long long acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (uint32_t j = threadIdx.x; j <= nsteps; j += blockDim.x) {
        for (uint32_t ph = 0; ph < 3; ph++) {
            const uint32_t pair = j < nsteps ? 3 * j + ph : (ph == 0 ? d.tspan_light : kNone);
            if (pair == kNone) continue;
            const unsigned long long a = d.tspan[2 * pair], b = d.tspan[2 * pair + 1];
            if (b != 0ull) {
                const int slot = j < nsteps ? (int)ph : 3;
                acc[slot] += b - ~a;
                acc[4 + slot] += 1ull;
                d.tspan[2 * pair] = 0ull;
                d.tspan[2 * pair + 1] = 0ull;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 8; q++) {
        unsigned long long v = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
        if ((threadIdx.x & 31u) == 0) red[q][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        unsigned long long t = 0;
        for (uint32_t w = 0; w < blockDim.x / 32; w++) t += red[threadIdx.x][w];
        d.tacc[threadIdx.x] += t;
    }
}

__global__ void chunk_end(Dev d, uint32_t steps) {
    pdl_prologue();
    *d.kbase += steps;
    *d.ev_n = 0;
}

namespace {

template <class... Args>
void launch_pdl(void (*kernel)(Args...), int grid, int block, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace

void launch_phase(const Dev &d, int phase, uint32_t koff, uint32_t kph, int grid, int block, cudaStream_t st) {
    // step_p2 walks short lists (crossers, intenders): half of step_p1's grid
    // each for the crossers and the intents (a quarter: 1.3% slower over the
    // regional day, the whole grid: 3% slower), one block for the intents at
    // stop-line cells (about a hundred per step at most), and one block per
    // `block` origin edges for the departure requests (at most one per origin
    // edge and step)
    const int g = (grid + 1) / 2;
    const uint32_t gdep = std::max(1u, (d.n_org + (uint32_t)block - 1) / (uint32_t)block);
#define LPSIM_PHASE(B)                                                                  \
    do {                                                                                \
        if (phase == 1) launch_pdl(step_p1<B>, grid, B, st, d, koff, kph);              \
        else launch_pdl(step_p2<B>, 2 * g + 1 + (int)gdep, B, st, d, koff, kph, (uint32_t)g, (uint32_t)g); \
    } while (0)
    switch (block) {
    case 128: LPSIM_PHASE(128); break;
    case 512: LPSIM_PHASE(512); break;
    default: LPSIM_PHASE(256); break;
    }
#undef LPSIM_PHASE
}

void launch_chunk_end(const Dev &d, uint32_t steps, cudaStream_t st) { launch_pdl(chunk_end, 1, 1, st, d, steps); }

void launch_apply_crossings(const Dev &d, int grid, cudaStream_t st) { apply_crossings<<<grid, 256, 0, st>>>(d); }

void launch_timing_fold(const Dev &d, uint32_t nsteps, cudaStream_t st) { timing_fold<<<1, 1024, 0, st>>>(d, nsteps); }

cudaError_t launch_small(const Dev &d, uint32_t k0, uint32_t nsteps, uint32_t *olist, uint32_t *no,
                         uint32_t map_words, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(no, 0, 4, st);
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)map_words * 16 * 5;
    if (smem > kSmallMapSmem) return cudaErrorInvalidValue;
    static bool attr_set = false;
    if (smem > 48 * 1024 && !attr_set) {
        e = cudaFuncSetAttribute(step_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmallMapSmem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    small_origins<<<(d.n_org + 255) / 256 + 1, 256, 0, st>>>(d, k0 + nsteps, olist, no);
    step_small<<<1, kSmallBlock, smem, st>>>(d, k0, nsteps, olist, no, map_words);
    return cudaGetLastError();
}

}  // namespace lpsim

namespace lpsim {

namespace {

// state of every live slot, scattered to vehicle-id order
__global__ void state_scatter(Dev d, uint32_t k, float *x, float *v, uint32_t *edge, uint8_t *lane, uint32_t *ridx) {
    const uint32_t n = *d.n_slots;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        if (d.s.flag[s] != kLive) continue;
        uint32_t id = d.s.id[s];
        x[id] = d.s.x[k & 1][s];
        v[id] = d.s.v[k & 1][s];
        edge[id] = d.route[d.s.es[s].rpos];
        lane[id] = d.s.lane[s];
        ridx[id] = d.s.es[s].rpos - d.roff[id];
    }
}

__global__ void max_arrival(Dev d, uint64_t n, uint32_t *out) {
    uint32_t best = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t a = d.arr[i];
        if (a != kNone && a > best) best = a;
    }
    best = __reduce_max_sync(0xFFFFFFFFu, best);
    if ((threadIdx.x & 31) == 0 && best) atomicMax(out, best);
}

}  // namespace

// bin-major [bin][edge] -> edge-major [edge][bin]
__global__ void transpose_bins(const uint32_t *in, uint32_t n_edges, uint32_t n_bins, uint32_t *out) {
    const size_t total = (size_t)n_edges * n_bins;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t e = i / n_bins, b = i % n_bins;
        out[i] = in[b * n_edges + e];
    }
}

void launch_transpose_bins(const uint32_t *in, uint32_t n_edges, uint32_t n_bins, uint32_t *out, cudaStream_t st) {
    transpose_bins<<<1024, 256, 0, st>>>(in, n_edges, n_bins, out);
}

void launch_route_records(const Dev &d, uint64_t n_trips, RouteRec *out, cudaStream_t st) {
    route_records<<<1024, 128, 0, st>>>(d, n_trips, out);
}

void launch_state_scatter(const Dev &d, uint32_t k, float *x, float *v, uint32_t *edge, uint8_t *lane,
                          uint32_t *ridx, cudaStream_t st) {
    state_scatter<<<256, 256, 0, st>>>(d, k, x, v, edge, lane, ridx);
}

void launch_max_arrival(const Dev &d, uint64_t n, uint32_t *out, cudaStream_t st) {
    max_arrival<<<256, 256, 0, st>>>(d, n, out);
}

}  // namespace lpsim
