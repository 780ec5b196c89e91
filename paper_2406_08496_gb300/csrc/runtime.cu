// Host runtime of liblpsim: the C ABI of include/lpsim.h.
//
// A context owns the device copy of the network (edge and node records,
// three rotating lane maps, two intent maps, the per-(edge, lane) claim
// slots), the trips in vehicle-id order (departure rank), the departure
// queues of the origin edges, two sets of vehicle slots (the compaction
// writes one set from the other), the link statistics and a few counters.
// Steps run as CUDA-graph chunks of `chunk_steps` steps (two step kernels
// per step plus a compaction, optionally a radix sort, every `sort_period`
// steps); steps that do not fill an aligned chunk are launched one by one.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/lpsim.h"
#include "ctx.h"
#include "host_par.h"
#include "lpsim_dev.cuh"

using namespace lpsim;

int lpsim_fail(int code, const std::string &msg);

namespace {

thread_local std::string g_last_error;
std::mutex g_alloc_mu;
void *(*g_alloc)(size_t, void *) = nullptr;
void (*g_release)(void *, void *) = nullptr;
void *g_alloc_user = nullptr;

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

#define CU(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(LPSIM_E_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

namespace {

template <class T>
int dnew(lpsim_ctx *c, T *&out, size_t count) {
    out = static_cast<T *>(c->dalloc(count * sizeof(T)));
    if (!out) return fail(LPSIM_E_OOM, "device allocation of " + std::to_string(count * sizeof(T)) + " bytes failed");
    return LPSIM_OK;
}

#define TRY(x)                 \
    do {                       \
        int rc_ = (x);         \
        if (rc_ != LPSIM_OK) return rc_; \
    } while (0)

// A device block held for the length of one call and given back, after the
// stream has finished with it, on every exit path.
struct Scratch {
    lpsim_ctx *c;
    void *p;
    Scratch(lpsim_ctx *ctx, size_t bytes) : c(ctx), p(ctx->dalloc(bytes)) {}
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
    ~Scratch() {
        if (!p) return;
        cudaStreamSynchronize(c->stream);
        auto it = std::find(c->blocks.begin(), c->blocks.end(), p);
        if (it != c->blocks.end()) c->blocks.erase(it);
        if (c->release) c->release(p, c->alloc_user);
        else cudaFree(p);
    }
};

// a device buffer whose contents change while stepping
template <class T>
int dnew_mut(lpsim_ctx *c, T *&out, size_t count) {
    int rc = dnew(c, out, count);
    if (rc == LPSIM_OK) c->mut.push_back({(void *)out, count * sizeof(T)});
    return rc;
}

int check_params(const lpsim_params *p) {
    if (!p) return fail(LPSIM_E_INVALID_ARG, "params is NULL");
    if (!(p->dt > 0.0f) || !(p->a > 0.0f) || !(p->b > 0.0f) || !(p->s0 >= 0.0f) || !(p->x0 > 0.0f) ||
        !std::isfinite(p->T) || !std::isfinite(p->g_a) || !std::isfinite(p->g_b) || !std::isfinite(p->alpha_i) ||
        !std::isfinite(p->alpha_a) || !std::isfinite(p->alpha_b) || !(p->eps_amp >= 0.0f) ||
        !(p->dlc_prob >= 0.0f && p->dlc_prob <= 1.0f) || !(p->dlc_gain >= 0.0f) || !std::isfinite(p->dlc_gain))
        return fail(LPSIM_E_INVALID_ARG, "model parameter out of range");
    if (p->bin_steps == 0 && p->n_bins != 0) return fail(LPSIM_E_INVALID_ARG, "n_bins without bin_steps");
    if (p->block_size && p->block_size != 128 && p->block_size != 256 && p->block_size != 512)
        return fail(LPSIM_E_INVALID_ARG, "block_size must be 0, 128, 256 or 512");
    if (p->flags & ~15u) return fail(LPSIM_E_INVALID_ARG, "unknown flag bits");
    if (p->sort_period > 256) return fail(LPSIM_E_INVALID_ARG, "sort_period must be at most 256");
    return LPSIM_OK;
}

int upload(lpsim_ctx *c, void *dst, const void *src, size_t bytes) {
    if (bytes) CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
    return LPSIM_OK;
}

int alloc_slots(lpsim_ctx *c, Slots &s, uint32_t cap) {
    // persistent fields (kept by snapshots)
    TRY(dnew_mut(c, s.es, cap));
    TRY(dnew_mut(c, s.id, cap));
    TRY(dnew_mut(c, s.rlast, cap));
    TRY(dnew_mut(c, s.tent, cap));
    TRY(dnew_mut(c, s.pcell, cap));
    TRY(dnew_mut(c, s.imark, cap));
    TRY(dnew_mut(c, s.lane, cap));
    TRY(dnew_mut(c, s.flag, cap));
    TRY(dnew_mut(c, s.tlc, cap));
    TRY(dnew_mut(c, s.cprev, cap));
    for (int i = 0; i < 2; i++) {
        TRY(dnew_mut(c, s.x[i], cap));
        TRY(dnew_mut(c, s.v[i], cap));
    }
    return LPSIM_OK;
}

// empty maps, waiting trips, cleared statistics, step 0
int reset_state(lpsim_ctx *c) {
    Dev &d = c->d;
    cudaStream_t st = c->stream;
    for (int i = 0; i < 3; i++) CU(cudaMemsetAsync(d.map[i], 0xFF, c->map_bytes, st));
    for (int i = 0; i < 2; i++) CU(cudaMemsetAsync(d.imap[i], 0, c->map_bytes, st));
    CU(cudaMemsetAsync(d.xreq, 0xFF, c->map_bytes, st));  // no request at any step
    for (int i = 0; i < 2; i++) CU(cudaMemsetAsync(d.claim[i], 0xFF, c->lane_slots * 4, st));
    CU(cudaMemsetAsync(d.ent, 0, c->n_edges * 8ull, st));
    CU(cudaMemsetAsync(d.ext, 0, c->n_edges * 8ull, st));
    CU(cudaMemsetAsync(d.tts, 0, c->n_edges * 8ull, st));
    size_t nb = (size_t)c->n_edges * c->p.n_bins * 4;
    if (nb) {
        CU(cudaMemsetAsync(d.bin_in, 0, nb, st));
        CU(cudaMemsetAsync(d.bin_tt, 0, nb, st));
        CU(cudaMemsetAsync(d.bin_cnt, 0, nb, st));
        CU(cudaMemsetAsync(d.bin_occ, 0, nb, st));
    }
    CU(cudaMemsetAsync(d.counts, 0, 8 * 4, st));
    CU(cudaMemsetAsync(d.kbase, 0, 4, st));
    CU(cudaMemsetAsync(d.n_slots, 0, 4, st));
    CU(cudaMemsetAsync(d.ev_n, 0, 4, st));
    CU(cudaMemsetAsync(d.ctr, 0, 8 * 8, st));
    CU(cudaMemsetAsync(d.err, 0, 4, st));
    if (c->loaded) {
        CU(cudaMemsetAsync(d.dep_act, 0xFF, c->n_trips * 4, st));
        CU(cudaMemsetAsync(d.arr, 0xFF, c->n_trips * 4, st));
        CU(cudaMemsetAsync(d.status, 0, c->n_trips, st));
        CU(cudaMemsetAsync(d.org_head, 0, (size_t)d.n_org * 4, st));
        CU(cudaMemsetAsync(d.dprev, 0xFF, (size_t)d.n_org * 4, st));
        CU(cudaMemcpyAsync(d.org_hd, c->org_hd0, (size_t)d.n_org * sizeof(QRec), cudaMemcpyDeviceToDevice, st));
    }
    c->k = 0;
    c->cur = 0;
    c->d.s = c->sets[0];
    c->stall_steps = 0;
    c->last_progress = 0;
    CU(cudaStreamSynchronize(st));
    return LPSIM_OK;
}

int read_status(lpsim_ctx *c) {
    // h_ctr: [0..7] counters, [8] err, [9] n_slots
    CU(cudaMemcpyAsync(c->h_ctr, c->d.ctr, 8 * 8, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(c->h_ctr + 8, c->d.err, 4, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(c->h_ctr + 9, c->d.n_slots, 4, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    uint32_t err = (uint32_t)(c->h_ctr[8] & 0xFFFFFFFFull);
    if (err & kErrCellTaken) return fail(LPSIM_E_INVARIANT, "two vehicles were written to one lane-map cell");
    if (err & kErrSlotOverflow) return fail(LPSIM_E_INVARIANT, "vehicle slot capacity exceeded");
    return LPSIM_OK;
}

// The kernels of step `koff` of a chunk (or of a direct step, koff = 0).
// Returns the slot set current after the step.  (With kernel timing on, the
// kernels stamp their own spans; nothing is inserted between them, so the
// graph keeps its programmatic dependent launches.)
int enqueue_step(lpsim_ctx *c, uint32_t koff, uint32_t kph, int cur, bool compact) {
    Dev d = c->d;
    d.s = c->sets[cur];
    for (int ph = 1; ph <= 2; ph++) launch_phase(d, ph, koff, kph, c->grid, c->block, c->stream);
    if (compact) {
        launch_compact(d, c->sets[cur ^ 1], c->w, koff, c->sort, c->grid, c->stream);
        cur ^= 1;
    }
    return cur;
}

// one step launched directly (kbase == k on entry; kbase == k+1 after)
int direct_step(lpsim_ctx *c) {
    bool compact = (c->k + 1) % c->R == 0;
    c->cur = enqueue_step(c, 0, (uint32_t)(c->k % 6), c->cur, compact);
    c->launches += 2;
    if (compact) c->launches += c->sort ? 3 + 3ull * ((c->w.key_bits + 7) / 8) + 1 : 3;
    launch_apply_crossings(c->d, c->grid, c->stream);
    launch_chunk_end(c->d, 1, c->stream);
    c->launches += 2;
    if (c->d.tspan) launch_timing_fold(c->d, 1, c->stream);
    CU(cudaGetLastError());
    c->k += 1;
    return LPSIM_OK;
}

int capture_chunk(lpsim_ctx *c, int start_set) {
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int cur = start_set;
    // a chunk always starts at a multiple of C, itself a multiple of 6
    for (uint32_t koff = 0; koff < c->C; koff++) cur = enqueue_step(c, koff, koff, cur, (koff + 1) % c->R == 0);
    launch_apply_crossings(c->d, c->grid, c->stream);
    launch_chunk_end(c->d, c->C, c->stream);
    if (c->d.tspan) launch_timing_fold(c->d, c->C, c->stream);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess) return fail(LPSIM_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->graph[start_set], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(LPSIM_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    if (cur != start_set) return fail(LPSIM_E_STATE, "chunk must hold an even number of compactions");
    return LPSIM_OK;
}

// kernels per chunk (for the launch counter)
uint64_t chunk_launches(const lpsim_ctx *c) {
    uint64_t per_compact = 3;
    if (c->sort) per_compact = 2 + 1 + 3ull * ((c->w.key_bits + 7) / 8) + 1;
    return 2ull * c->C + (c->C / c->R) * per_compact + 2;
}

int chunk(lpsim_ctx *c) {
    if (c->C % 6 != 0 || c->k % c->C != 0) return fail(LPSIM_E_STATE, "graph chunk not aligned to a multiple of 6 steps");
    if (!c->graph[c->cur]) TRY(capture_chunk(c, c->cur));
    CU(cudaGraphLaunch(c->graph[c->cur], c->stream));
    c->launches += chunk_launches(c);
    c->k += c->C;
    return LPSIM_OK;
}

// Light load: at most light_trips trips can be on the network or waiting in
// the chunk starting at step k (trips due before its end minus those arrived;
// h_ctr is current).
bool light_chunk_ok(const lpsim_ctx *c) {
    if (c->p.flags & LPSIM_F_NO_LIGHT) return false;
    const uint64_t due = (uint64_t)(std::lower_bound(c->dep_sorted.begin(), c->dep_sorted.end(), c->k + c->C) -
                                    c->dep_sorted.begin());
    return due <= c->h_ctr[1] + (c->p.light_trips ? c->p.light_trips : kSmallMax);
}

// One chunk in the light-load kernel, then the compaction that closes every
// chunk and the step-counter update.
int light_chunk(lpsim_ctx *c) {
    Dev d = c->d;
    d.s = c->sets[c->cur];
    // with LPSIM_F_SHARED_MAPS the lane maps of a small network ride in the
    // light-load kernel's shared memory for the chunk
    const uint64_t words = (c->map_bytes + 15) / 16;
    const uint32_t map_words =
        ((c->p.flags & LPSIM_F_SHARED_MAPS) && words * 16 * 5 <= kSmallMapSmem) ? (uint32_t)words : 0u;
    CU(launch_small(d, c->k, c->C, c->small_list, c->small_n, map_words, c->stream));
    launch_compact(d, c->sets[c->cur ^ 1], c->w, c->C - 1, c->sort, c->grid, c->stream);
    c->cur ^= 1;
    launch_apply_crossings(c->d, c->grid, c->stream);
    launch_chunk_end(c->d, c->C, c->stream);
    if (c->d.tspan) launch_timing_fold(c->d, c->C, c->stream);
    CU(cudaGetLastError());
    c->launches += 4 + (c->sort ? 3 + 3ull * ((c->w.key_bits + 7) / 8) + 1 : 3);
    c->light_chunks++;
    c->k += c->C;
    return LPSIM_OK;
}

// Run up to n steps; stop early once every trip has arrived (if stop_done).
// Returns steps actually taken in *taken.
int run_steps(lpsim_ctx *c, uint64_t n, bool stop_done, uint64_t *taken) {
    const uint32_t k0 = c->k;
    uint64_t left = n;
    TRY(read_status(c));
    while (left > 0) {
        if (stop_done) {
            TRY(read_status(c));
            if (c->h_ctr[1] >= c->n_trips) break;
        }
        uint64_t before = c->k;
        if (c->k % c->C == 0 && left >= c->C) {
            if (light_chunk_ok(c))
                TRY(light_chunk(c));
            else
                TRY(chunk(c));
        } else {
            uint32_t todo = (uint32_t)std::min<uint64_t>(left, c->k % c->C == 0 ? left : c->C - c->k % c->C);
            for (uint32_t j = 0; j < todo; j++) TRY(direct_step(c));
        }
        left -= c->k - before;
        const unsigned long long prog_before = c->last_progress;
        TRY(read_status(c));
        // gridlock watch: vehicles on the network and no crossing, departure or arrival
        unsigned long long prog = c->h_ctr[1] + c->h_ctr[3];
        unsigned long long active = c->h_ctr[4] - c->h_ctr[1];
        // Idle network: a whole chunk passed with no vehicle on the network and
        // nothing departing or arriving, so every map, claim and mark is clear
        // and every trip due so far has arrived.  The steps until the next
        // departure change nothing: jump to the chunk that holds it.
        if (active == 0 && prog == prog_before && c->k % c->C == 0 && c->k - before == c->C && left > 0) {
            auto nx = std::lower_bound(c->dep_sorted.begin(), c->dep_sorted.end(), c->k);
            if (nx != c->dep_sorted.end()) {
                const uint64_t target = std::min<uint64_t>((uint64_t)(*nx / c->C) * c->C, c->k + left / c->C * c->C);
                if (target > c->k) {
                    left -= target - c->k;
                    c->k = (uint32_t)target;
                    c->skipped += target - before - c->C;
                    CU(cudaMemcpyAsync(c->d.kbase, &c->k, 4, cudaMemcpyHostToDevice, c->stream));
                    CU(cudaStreamSynchronize(c->stream));
                }
            }
        }
        if (prog != c->last_progress || active == 0) {
            c->last_progress = prog;
            c->stall_steps = 0;
        } else {
            c->stall_steps += c->k - before;
            if (c->p.gridlock_steps && c->stall_steps >= c->p.gridlock_steps)
                return fail(LPSIM_E_GRIDLOCK, "no vehicle crossed, departed or arrived for " +
                                                  std::to_string(c->stall_steps) + " steps");
        }
        if (stop_done && c->h_ctr[1] >= c->n_trips) break;
    }
    if (stop_done) {
        TRY(read_status(c));
        if (c->h_ctr[1] >= c->n_trips && c->n_trips > 0) {
            // the last chunk may have run past the last arrival; nothing moves
            // after it, so only the step counter needs to come back
            CU(cudaMemsetAsync(c->d_tmp, 0, 4, c->stream));
            launch_max_arrival(c->d, c->n_trips, c->d_tmp, c->stream);
            uint32_t kfin = 0;
            CU(cudaMemcpyAsync(&kfin, c->d_tmp, 4, cudaMemcpyDeviceToHost, c->stream));
            CU(cudaStreamSynchronize(c->stream));
            if (kfin < c->k && kfin >= k0) {
                c->k = kfin;
                CU(cudaMemcpyAsync(c->d.kbase, &c->k, 4, cudaMemcpyHostToDevice, c->stream));
                CU(cudaStreamSynchronize(c->stream));
            } else if (kfin < k0) {
                c->k = std::max(c->k, k0);
            }
        }
    }
    *taken = c->k - k0;
    return LPSIM_OK;
}

}  // namespace

int lpsim_fail(int code, const std::string &msg) { return fail(code, msg); }

extern "C" {

const char *lpsim_last_error(void) { return g_last_error.c_str(); }

const char *lpsim_version(void) { return "lpsim-gb300 1.0 (sm_103a)"; }

int lpsim_set_allocator(void *(*alloc)(size_t, void *), void (*release)(void *, void *), void *user) {
    if ((alloc == nullptr) != (release == nullptr)) return fail(LPSIM_E_INVALID_ARG, "give both callbacks or neither");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc;
    g_release = release;
    g_alloc_user = user;
    return LPSIM_OK;
}

}  // extern "C"

namespace {

int load_network_impl(lpsim_ctx **out, const lpsim_network *net, const lpsim_params *p, void *stream) {
    if (!out) return fail(LPSIM_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    TRY(check_params(p));
    if (!net || !net->edge_src || !net->edge_dst || !net->edge_len_m || !net->edge_lanes || !net->edge_vmax ||
        !net->node_green_steps)
        return fail(LPSIM_E_INVALID_ARG, "network array is NULL");
    const uint32_t nn = net->n_nodes, ne = net->n_edges;
    if (nn == 0 || ne == 0) return fail(LPSIM_E_INVALID_ARG, "empty network");
    std::vector<uint32_t> n_in(nn, 0), n_out(nn, 0);
    std::vector<uint8_t> orank(ne), arank(ne);
    std::vector<EdgeRec> er(ne);
    std::vector<uint32_t> slot_off(ne);
    std::vector<uint16_t> lens(ne);
    std::vector<uint32_t> moffs(ne);
    uint64_t cells = 0, slots = 0, canon = 0;
    for (uint32_t e = 0; e < ne; e++) {
        if (net->edge_src[e] >= nn || net->edge_dst[e] >= nn)
            return fail(LPSIM_E_INVALID_ARG, "edge " + std::to_string(e) + ": node id out of range");
        if (net->edge_lanes[e] < 1 || net->edge_lanes[e] > 4)
            return fail(LPSIM_E_INVALID_ARG, "edge " + std::to_string(e) + ": lanes must be 1..4");
        float L = net->edge_len_m[e];
        if (!(L > 0.0f) || !(L <= 65535.0f))
            return fail(LPSIM_E_INVALID_ARG, "edge " + std::to_string(e) + ": length must be in (0, 65535] m");
        float vm = net->edge_vmax[e];
        if (!(vm > 0.0f) || !(vm <= 254.0f))
            return fail(LPSIM_E_INVALID_ARG, "edge " + std::to_string(e) + ": speed limit must be in (0, 254] m/s");
        uint32_t len = (uint32_t)std::ceil(L);
        if (len < 1) len = 1;
        orank[e] = (uint8_t)n_out[net->edge_src[e]];
        if (++n_out[net->edge_src[e]] > 255) return fail(LPSIM_E_INVALID_ARG, "node with more than 255 out-edges");
        uint32_t rank = n_in[net->edge_dst[e]];
        if (++n_in[net->edge_dst[e]] > 255) return fail(LPSIM_E_INVALID_ARG, "node with more than 255 in-edges");
        arank[e] = net->edge_approach_rank ? net->edge_approach_rank[e] : (uint8_t)rank;
        lens[e] = (uint16_t)len;
        moffs[e] = (uint32_t)cells;
        er[e].moff = (uint32_t)cells;
        er[e].len = (uint16_t)len;
        er[e].lanes = net->edge_lanes[e];
        er[e].v0 = vm;
        er[e].dst = net->edge_dst[e];
        cells += (uint64_t)row_stride(len) * net->edge_lanes[e];
        canon += (uint64_t)len * net->edge_lanes[e];
        slot_off[e] = (uint32_t)slots;
        slots += net->edge_lanes[e];
        if (cells >= 0xFFFFFFF0ull) return fail(LPSIM_E_INVALID_ARG, "lane map larger than 4 GiB");
    }
    std::vector<NodeRec> nr(nn);
    for (uint32_t i = 0; i < nn; i++) {
        nr[i].green = net->node_green_steps[i];
        nr[i].nphase = 0;
        nr[i].nout = (uint8_t)n_out[i];
        nr[i].pad = 0;
    }
    for (uint32_t e = 0; e < ne; e++) {
        uint32_t node = net->edge_dst[e];
        if (arank[e] >= n_in[node])
            return fail(LPSIM_E_INVALID_ARG, "edge " + std::to_string(e) + ": approach rank not below in-degree");
        er[e].arank = arank[e];
        if ((uint32_t)arank[e] + 1 > nr[node].nphase) nr[node].nphase = (uint8_t)(arank[e] + 1);
    }

    lpsim_ctx *c = new (std::nothrow) lpsim_ctx();
    if (!c) return fail(LPSIM_E_OOM, "host allocation failed");
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        c->alloc = g_alloc;
        c->release = g_release;
        c->alloc_user = g_alloc_user;
    }
    auto bail = [&](int rc) {
        delete c;
        return rc;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) return bail(fail(LPSIM_E_CUDA, "no CUDA device"));
    cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
    c->stream = static_cast<cudaStream_t>(stream);
    if (!c->stream) {
        // graph capture needs a stream other than the legacy default stream
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(fail(LPSIM_E_CUDA, "cannot create a stream"));
        c->own_stream = true;
    }
    c->p = *p;
    c->n_nodes = nn;
    c->n_edges = ne;
    c->moff = moffs;
    c->len = lens;
    c->lanes.assign(net->edge_lanes, net->edge_lanes + ne);
    c->src.assign(net->edge_src, net->edge_src + ne);
    c->dst.assign(net->edge_dst, net->edge_dst + ne);
    c->map_bytes = cells + 16;
    c->canon_cells = canon;
    c->lane_slots = slots;
    c->R = p->sort_period ? p->sort_period : 256;
    uint32_t base = 2 * c->R;
    base = base % 3 == 0 ? base : base * 3;  // chunk = multiple of 2R and of 3 (lane-map rotation)
    uint32_t want = p->chunk_steps ? p->chunk_steps : 1536;
    c->C = std::max(base, (want + base - 1) / base * base);
    c->block = p->block_size ? (int)p->block_size : 256;
    c->grid = c->n_sm * (int)(p->blocks_per_sm ? p->blocks_per_sm : 4) * 256 / c->block;
    if (c->grid < 1) c->grid = 1;
    c->sort = (p->flags & 1u) == 0;
    c->d.check = (p->flags & 2u) ? 1u : 0u;

    Dev &d = c->d;
    d.m.dt = p->dt;
    d.m.a = p->a;
    d.m.s0 = p->s0;
    d.m.T = p->T;
    d.m.two_sqrt_ab = (float)(2.0 * std::sqrt((double)p->a * (double)p->b));
    d.m.x0 = p->x0;
    d.m.g_a = p->g_a;
    d.m.g_b = p->g_b;
    d.m.alpha_i = p->alpha_i;
    d.m.alpha_a = p->alpha_a;
    d.m.alpha_b = p->alpha_b;
    d.m.eps_amp = p->eps_amp;
    d.m.seed = p->seed;
    d.m.bin_steps = p->bin_steps;
    d.m.n_bins = p->n_bins;
    d.m.dlc_prob = p->dlc_prob;
    d.m.dlc_gain = p->dlc_gain;
    d.n_edges = ne;

    EdgeRec *edge = nullptr;
    NodeRec *node = nullptr;
    uint32_t *so = nullptr;
    uint8_t *ork = nullptr;
    int rc;
    if ((rc = dnew(c, edge, ne)) || (rc = dnew(c, node, nn)) || (rc = dnew(c, so, ne)) || (rc = dnew(c, ork, ne)))
        return bail(rc);
    d.edge = edge;
    d.node = node;
    d.slot_off = so;
    d.orank = ork;
    for (int i = 0; i < 3; i++)
        if ((rc = dnew_mut(c, d.map[i], c->map_bytes))) return bail(rc);
    for (int i = 0; i < 2; i++)
        if ((rc = dnew_mut(c, d.imap[i], c->map_bytes))) return bail(rc);
    // one crossing-request record per 16 map bytes: every lane row starts on
    // a 16-byte boundary and spans at least 16 bytes
    if ((rc = dnew_mut(c, d.xreq, c->map_bytes / 16)) || (rc = dnew_mut(c, d.snap, 2))) return bail(rc);
    if ((rc = dnew_mut(c, d.claim[0], slots)) || (rc = dnew_mut(c, d.claim[1], slots)) ||
        (rc = dnew_mut(c, d.ent, ne)) || (rc = dnew_mut(c, d.ext, ne)) || (rc = dnew_mut(c, d.tts, ne)))
        return bail(rc);
    size_t nb = (size_t)ne * p->n_bins;
    if ((rc = dnew_mut(c, d.bin_in, nb)) || (rc = dnew_mut(c, d.bin_tt, nb)) || (rc = dnew_mut(c, d.bin_cnt, nb)) ||
        (rc = dnew_mut(c, d.bin_occ, nb)))
        return bail(rc);
    if ((rc = dnew_mut(c, d.counts, 8)) || (rc = dnew_mut(c, d.kbase, 1)) || (rc = dnew_mut(c, d.n_slots, 1)) ||
        (rc = dnew_mut(c, d.ev_n, 1)) ||
        (rc = dnew_mut(c, d.ctr, 8)) || (rc = dnew_mut(c, d.err, 1)) || (rc = dnew(c, c->d_tmp, 4)))
        return bail(rc);
    if (cudaMallocHost(&c->h_ctr, 16 * 8) != cudaSuccess) return bail(fail(LPSIM_E_OOM, "pinned allocation failed"));
    if ((rc = upload(c, edge, er.data(), ne * sizeof(EdgeRec))) || (rc = upload(c, node, nr.data(), nn * sizeof(NodeRec))) ||
        (rc = upload(c, so, slot_off.data(), ne * 4)) || (rc = upload(c, ork, orank.data(), ne)))
        return bail(rc);
    // key bits of the radix sort: enough for every lane-map cell index
    uint32_t bits = 1;
    while (bits < 32 && (1ull << bits) < c->map_bytes) bits++;
    c->w.key_bits = bits;
    if ((rc = reset_state(c))) return bail(rc);
    c->scen_node_off = {0, nn};
    c->scen_edge_off = {0, ne};
    c->scen_cell_off = {0, canon};
    *out = c;
    return LPSIM_OK;
}

}  // namespace

extern "C" {

int lpsim_load_network(lpsim_ctx **out, const lpsim_network *net, const lpsim_params *p, void *stream) {
    return load_network_impl(out, net, p, stream);
}

int lpsim_load_network_batch(lpsim_ctx **out, uint32_t n_scen, const lpsim_network *nets, const lpsim_params *p,
                             void *stream) {
    if (!out) return fail(LPSIM_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_scen == 0 || !nets) return fail(LPSIM_E_INVALID_ARG, "no scenarios");
    uint64_t nn = 0, ne = 0;
    bool any_rank = false;
    for (uint32_t sc = 0; sc < n_scen; sc++) {
        const lpsim_network &g = nets[sc];
        if (!g.edge_src || !g.edge_dst || !g.edge_len_m || !g.edge_lanes || !g.edge_vmax || !g.node_green_steps)
            return fail(LPSIM_E_INVALID_ARG, "scenario " + std::to_string(sc) + ": network array is NULL");
        nn += g.n_nodes;
        ne += g.n_edges;
        any_rank |= g.edge_approach_rank != nullptr;
    }
    if (nn >= 0xFFFFFFF0ull || ne >= 0xFFFFFFF0ull) return fail(LPSIM_E_INVALID_ARG, "batch too large");
    std::vector<uint32_t> src(ne), dst(ne), green(nn);
    std::vector<float> len(ne), vmax(ne);
    std::vector<uint8_t> lanes(ne), rank(any_rank ? ne : 0);
    std::vector<uint64_t> noff{0}, eoff{0}, coff{0};
    uint64_t no = 0, eo = 0, cells = 0;
    for (uint32_t sc = 0; sc < n_scen; sc++) {
        const lpsim_network &g = nets[sc];
        std::vector<uint32_t> n_in(g.n_nodes, 0);
        for (uint32_t e = 0; e < g.n_edges; e++) {
            if (g.edge_src[e] >= g.n_nodes || g.edge_dst[e] >= g.n_nodes)
                return fail(LPSIM_E_INVALID_ARG, "scenario " + std::to_string(sc) + ": node id out of range");
            src[eo + e] = (uint32_t)(g.edge_src[e] + no);
            dst[eo + e] = (uint32_t)(g.edge_dst[e] + no);
            len[eo + e] = g.edge_len_m[e];
            vmax[eo + e] = g.edge_vmax[e];
            lanes[eo + e] = g.edge_lanes[e];
            uint32_t r = n_in[g.edge_dst[e]]++;
            if (any_rank) rank[eo + e] = g.edge_approach_rank ? g.edge_approach_rank[e] : (uint8_t)r;
            cells += (uint64_t)std::max(1.0f, std::ceil(g.edge_len_m[e])) * g.edge_lanes[e];
        }
        for (uint32_t i = 0; i < g.n_nodes; i++) green[no + i] = g.node_green_steps[i];
        no += g.n_nodes;
        eo += g.n_edges;
        noff.push_back(no);
        eoff.push_back(eo);
        coff.push_back(cells);
    }
    lpsim_network u{(uint32_t)nn, (uint32_t)ne, src.data(), dst.data(), len.data(), lanes.data(), vmax.data(),
                    green.data(), any_rank ? rank.data() : nullptr};
    TRY(load_network_impl(out, &u, p, stream));
    (*out)->scen_node_off = noff;
    (*out)->scen_edge_off = eoff;
    (*out)->scen_cell_off = coff;
    return LPSIM_OK;
}

int lpsim_batch_offsets(lpsim_ctx *c, uint32_t n_scen, uint64_t *node_off, uint64_t *edge_off, uint64_t *cell_off,
                        uint64_t *trip_off) {
    if (!c) return fail(LPSIM_E_INVALID_ARG, "ctx is NULL");
    if (c->scen_edge_off.size() != (size_t)n_scen + 1) return fail(LPSIM_E_INVALID_ARG, "n_scen does not match");
    for (uint32_t i = 0; i <= n_scen; i++) {
        if (node_off) node_off[i] = c->scen_node_off[i];
        if (edge_off) edge_off[i] = c->scen_edge_off[i];
        if (cell_off) cell_off[i] = c->scen_cell_off[i];
        if (trip_off) trip_off[i] = c->scen_trip_off.size() == (size_t)n_scen + 1 ? c->scen_trip_off[i] : 0;
    }
    return LPSIM_OK;
}

}  // extern "C"

namespace {

// Trips of one simulation or of a batch of scenarios.  scen (nullable): the
// scenario of each input trip, non-decreasing; seeds (nullable): the
// lane-change seed of each scenario (default: the context's seed).
// Host staging of the id-ordered routes, kept for the process between demand
// loads: a fresh buffer's pages fault in at first touch (about 50 ms for the
// 1.4 GB of the 2.82M-trip day), and the assignment loop loads a demand per
// simulation.  One load holds it at a time (others allocate their own); it
// grows to the largest demand seen and is never shrunk.
struct RouteStaging {
    std::mutex mu;
    std::unique_ptr<uint32_t[]> buf;
    uint64_t cap = 0;
    bool busy = false;
};

RouteStaging &route_staging() {
    static RouteStaging s;
    return s;
}

// the staging for one load: the process's buffer when free, else a private one
struct RouteBuffer {
    uint32_t *p = nullptr;
    bool pooled = false;
    std::unique_ptr<uint32_t[]> own;
    explicit RouteBuffer(uint64_t n) {
        RouteStaging &st = route_staging();
        {
            std::lock_guard<std::mutex> g(st.mu);
            if (!st.busy) {
                if (st.cap < n) {
                    st.buf.reset();
                    st.buf.reset(new (std::nothrow) uint32_t[n]);
                    st.cap = st.buf ? n : 0;
                }
                if (st.buf) {
                    st.busy = true;
                    pooled = true;
                    p = st.buf.get();
                }
            }
        }
        if (!pooled) {
            own.reset(new (std::nothrow) uint32_t[n]);
            p = own.get();
        }
    }
    RouteBuffer(const RouteBuffer &) = delete;
    RouteBuffer &operator=(const RouteBuffer &) = delete;
    ~RouteBuffer() {
        if (!pooled) return;
        RouteStaging &st = route_staging();
        std::lock_guard<std::mutex> g(st.mu);
        st.busy = false;
    }
};

int load_demand_impl(lpsim_ctx *c, uint64_t n, const uint32_t *depart_step, const uint64_t *route_off,
                     const uint32_t *route_edges, uint32_t *out_vid, const uint32_t *scen, uint32_t n_scen,
                     const uint64_t *seeds, const uint8_t *vtype = nullptr) {
    if (!c) return fail(LPSIM_E_INVALID_ARG, "ctx is NULL");
    if (c->loaded) return fail(LPSIM_E_STATE, "demand already loaded");
    // n == 0 is a valid (empty) demand: every step finds nothing to move and
    // lpsim_run returns at once
    if (!route_off || (n > 0 && (!depart_step || !route_edges)))
        return fail(LPSIM_E_INVALID_ARG, "trip array is NULL");
    if (n >= 0xFFFFFFF0ull) return fail(LPSIM_E_INVALID_ARG, "too many trips");
    if (route_off[0] != 0) return fail(LPSIM_E_INVALID_ARG, "route_off[0] must be 0");
    // Checks, spread over the host's threads; the lowest failing trip is
    // reported (offsets first, then edges, as a sequential pass would).
    {
        std::mutex mu;
        uint64_t bad = n;
        parallel_pieces(n, [&](uint64_t j0, uint64_t j1, uint64_t) {
            for (uint64_t j = j0; j < j1; j++)
                if (route_off[j + 1] <= route_off[j]) {
                    std::lock_guard<std::mutex> g(mu);
                    bad = std::min(bad, j);
                    return;
                }
        });
        if (bad < n)
            return fail(LPSIM_E_INVALID_ARG, "trip " + std::to_string(bad) + ": empty route or route_off not increasing");
    }
    const uint64_t total = route_off[n];
    if (total >= 0xFFFFFFF0ull) return fail(LPSIM_E_INVALID_ARG, "total route length must stay below 2^32");
    if (vtype) {
        const uint32_t nt = (uint32_t)std::max<size_t>(c->types.size(), 1);
        for (uint64_t j = 0; j < n; j++)
            if (vtype[j] >= nt)
                return fail(LPSIM_E_INVALID_ARG, "trip " + std::to_string(j) + ": vehicle type out of range");
    }
    {
        std::mutex mu;
        uint64_t bad = n;
        int kind = 0;
        const uint32_t ne = c->n_edges;
        // each edge's (tail, head) in one record: one random read per route entry
        std::vector<uint2> ends(ne);
        parallel_pieces(ne, [&](uint64_t e0, uint64_t e1, uint64_t) {
            for (uint64_t e = e0; e < e1; e++) ends[e] = make_uint2(c->src[e], c->dst[e]);
        });
        parallel_pieces(n, [&](uint64_t j0, uint64_t j1, uint64_t) {
            for (uint64_t j = j0; j < j1; j++) {
                int k = 0;
                uint32_t head = 0;  // head node of the previous edge of the route
                for (uint64_t q = route_off[j]; q < route_off[j + 1]; q++) {
                    const uint32_t e = route_edges[q];
                    if (e >= ne) {
                        k = 1;
                        break;
                    }
                    const uint2 te = ends[e];
                    if (q > route_off[j] && head != te.x) {
                        k = 2;
                        break;
                    }
                    head = te.y;
                }
                if (k) {
                    std::lock_guard<std::mutex> g(mu);
                    if (j < bad) {
                        bad = j;
                        kind = k;
                    }
                    return;
                }
            }
        });
        if (bad < n)
            return fail(LPSIM_E_INVALID_ARG, "trip " + std::to_string(bad) + (kind == 1 ? ": edge id out of range"
                                                                                  : ": route edges are not contiguous"));
    }
    // vehicle ids: stable sort by departure step (a counting sort when the
    // steps span less than 2^24)
    std::vector<uint32_t> order(n);
    const uint32_t max_dep = n ? *std::max_element(depart_step, depart_step + n) : 0u;
    if (max_dep < (1u << 24)) {
        std::vector<uint64_t> pos((size_t)max_dep + 2, 0);
        for (uint64_t j = 0; j < n; j++) pos[(size_t)depart_step[j] + 1]++;
        for (size_t t = 1; t < pos.size(); t++) pos[t] += pos[t - 1];
        for (uint64_t j = 0; j < n; j++) order[pos[depart_step[j]]++] = (uint32_t)j;
    } else {
        std::iota(order.begin(), order.end(), 0u);
        std::stable_sort(order.begin(), order.end(),
                         [&](uint32_t a, uint32_t b) { return depart_step[a] < depart_step[b]; });
    }
    std::vector<uint32_t> dep(n), roff(n + 1);
    // the routes in vehicle-id order, in the process's staging buffer (never
    // cleared: every entry is written below, by the host's threads)
    const uint64_t rsize = total ? total : 1;
    RouteBuffer rbuf(rsize);
    uint32_t *const route = rbuf.p;
    if (!route) return fail(LPSIM_E_OOM, "host allocation of the route array failed");
    if (!total) route[0] = 0;
    // lane-change draw keys: seed ^ (id within the scenario) * C1; a single
    // scenario's key follows from the id on the device
    std::vector<uint64_t> hkey(scen ? n : 0);
    if (scen) {
        std::vector<uint64_t> local(std::max<uint32_t>(n_scen, 1u), 0);
        for (uint64_t id = 0; id < n; id++) {
            const uint32_t j = order[id];
            hkey[id] = (seeds ? seeds[scen[j]] : c->p.seed) ^ (local[scen[j]]++ * 0x9E3779B97F4A7C15ull);
        }
    }
    // per id (gathers spread over the host's threads): departure step, route
    // length, first edge, vehicle type; the route offsets are their prefix sum
    std::vector<uint32_t> first(n);
    const bool typed = !c->types.empty();
    std::vector<uint8_t> vt(typed ? n : 0);
    parallel_pieces(n, [&](uint64_t i0, uint64_t i1, uint64_t) {
        for (uint64_t id = i0; id < i1; id++) {
            const uint32_t j = order[id];
            dep[id] = depart_step[j];
            roff[id + 1] = (uint32_t)(route_off[j + 1] - route_off[j]);
            first[id] = route_edges[route_off[j]];
            if (typed) vt[id] = vtype ? vtype[j] : (uint8_t)0;
            if (out_vid) out_vid[j] = (uint32_t)id;
        }
    });
    roff[0] = 0;
    for (uint64_t id = 0; id < n; id++) roff[id + 1] += roff[id];
    parallel_pieces(n, [&](uint64_t i0, uint64_t i1, uint64_t) {
        for (uint64_t id = i0; id < i1; id++) {
            const uint32_t j = order[id];
            std::memcpy(route + roff[id], route_edges + route_off[j], (size_t)(roff[id + 1] - roff[id]) * 4);
        }
    });
    c->dep_sorted = dep;  // nondecreasing: ids are ranks by departure step
    // departure queues: ids grouped by first edge, ascending within a group
    std::vector<uint32_t> cnt(c->n_edges + 1, 0);
    for (uint64_t id = 0; id < n; id++) cnt[first[id] + 1]++;
    std::vector<uint32_t> org_edge, org_qoff, org_qend;
    for (uint32_t e = 0; e < c->n_edges; e++) {
        if (cnt[e + 1]) {
            org_edge.push_back(e);
            org_qoff.push_back(cnt[e]);
            org_qend.push_back(cnt[e] + cnt[e + 1]);
        }
        cnt[e + 1] += cnt[e];
    }
    std::vector<uint32_t> qid(n);
    {
        std::vector<uint32_t> fill(cnt.begin(), cnt.end() - 1);
        for (uint64_t id = 0; id < n; id++) qid[fill[first[id]]++] = (uint32_t)id;
    }
    Dev &d = c->d;
    const uint32_t norg = (uint32_t)org_edge.size();
    // queue records (vehicle, departure step, route span) in queue order
    std::vector<QRec> qrec(n), hd0(norg);
    parallel_pieces(n, [&](uint64_t q0, uint64_t q1, uint64_t) {
        for (uint64_t q = q0; q < q1; q++) qrec[q] = QRec{qid[q], dep[qid[q]], roff[qid[q]], roff[qid[q] + 1]};
    });
    std::vector<EdgeRec> orec(norg);
    {
        std::vector<EdgeRec> all(c->n_edges);
        CU(cudaMemcpy(all.data(), d.edge, c->n_edges * sizeof(EdgeRec), cudaMemcpyDeviceToHost));
        for (uint32_t j = 0; j < norg; j++) {
            orec[j] = all[org_edge[j]];
            hd0[j] = qrec[org_qoff[j]];
        }
    }
    uint32_t *droute, *droff, *oe, *oq, *oqe;
    uint64_t *dhkey;
    QRec *dqrec;
    EdgeRec *dorec;
    RouteRec *drrec;
    dhkey = nullptr;
    if (scen) TRY(dnew(c, dhkey, n));
    TRY(dnew(c, droute, rsize));
    TRY(dnew(c, droff, n + 1));
    TRY(dnew(c, drrec, rsize));
    TRY(dnew_mut(c, d.dep_act, n));
    TRY(dnew_mut(c, d.arr, n));
    TRY(dnew_mut(c, d.status, n));
    TRY(dnew(c, oe, norg));
    TRY(dnew(c, oq, norg));
    TRY(dnew(c, oqe, norg));
    TRY(dnew(c, dqrec, n));
    TRY(dnew(c, dorec, norg));
    TRY(dnew_mut(c, d.org_head, norg));
    TRY(dnew_mut(c, d.org_hd, norg));
    TRY(dnew(c, c->org_hd0, norg));
    TRY(dnew_mut(c, d.dprev, norg));
    for (int i = 0; i < 2; i++) TRY(dnew(c, d.dep_rec[i], norg));
    // crossing log: room for a chunk at the busiest hour of a day (past it the
    // step kernels update the statistics directly)
    d.ev_cap = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(4ull * n, 1ull << 20), 1ull << 25);
    TRY(dnew(c, d.ev_log, d.ev_cap));
    TRY(dnew(c, c->small_list, std::max<uint32_t>(norg, 1u)));
    TRY(dnew(c, c->small_n, 4));
    // slots: live vehicles plus the holes left between compactions by
    // arrivals and by departures that lost an entry conflict
    const uint64_t cap64 = n + 256ull * norg + 1024;
    if (cap64 >= 0xFFFFFFF0ull) return fail(LPSIM_E_INVALID_ARG, "too many trips for the slot index");
    const uint32_t cap = (uint32_t)cap64;
    for (int i = 0; i < 2; i++) TRY(alloc_slots(c, c->sets[i], cap));
    for (int i = 0; i < 2; i++) {
        TRY(dnew(c, d.cross_list[i], cap));
        TRY(dnew(c, d.intend_list[i], cap));
    }
    uint32_t max_tiles = (cap + compact_tile() - 1) / compact_tile() + 1;
    c->w.max_tiles = max_tiles;
    TRY(dnew(c, c->w.tile_cnt, max_tiles));
    TRY(dnew(c, c->w.tile_off, max_tiles + 2));
    TRY(dnew(c, c->w.hist, 256ull * max_tiles));
    for (int i = 0; i < 2; i++) {
        TRY(dnew(c, c->w.key[i], cap));
        TRY(dnew(c, c->w.perm[i], cap));
    }
    if (scen) TRY(upload(c, dhkey, hkey.data(), n * 8));
    if (typed) {
        std::vector<TypeRec> tr(kMaxTypes);
        for (size_t t = 0; t < c->types.size(); t++) {
            const lpsim_vehicle_type &y = c->types[t];
            tr[t] = TypeRec{y.a, y.s0, y.T, (float)(2.0 * std::sqrt((double)y.a * (double)y.b)), y.vmax, {0, 0, 0}};
        }
        TypeRec *dtr = nullptr;
        uint8_t *dvt = nullptr;
        TRY(dnew(c, dtr, kMaxTypes));
        TRY(dnew(c, dvt, n));
        TRY(upload(c, dtr, tr.data(), kMaxTypes * sizeof(TypeRec)));
        TRY(upload(c, dvt, vt.data(), n));
        d.types = dtr;
        d.trip_vt = dvt;
        d.typed = 1;
    }
    TRY(upload(c, droute, route, rsize * 4));
    TRY(upload(c, droff, roff.data(), (n + 1) * 4));
    TRY(upload(c, oe, org_edge.data(), norg * 4ull));
    TRY(upload(c, oq, org_qoff.data(), norg * 4ull));
    TRY(upload(c, oqe, org_qend.data(), norg * 4ull));
    TRY(upload(c, dqrec, qrec.data(), n * sizeof(QRec)));
    TRY(upload(c, dorec, orec.data(), norg * sizeof(EdgeRec)));
    TRY(upload(c, c->org_hd0, hd0.data(), norg * sizeof(QRec)));
    d.hkey = dhkey;
    d.hkey_from_id = scen ? 0u : 1u;
    d.route = droute;
    d.roff = droff;
    d.rrec = drrec;
    d.n_org = norg;
    d.org_edge = oe;
    d.org_qoff = oq;
    d.org_qend = oqe;
    d.qrec = dqrec;
    d.org_rec = dorec;
    d.cap = cap;
    launch_route_records(d, n, drrec, c->stream);
    CU(cudaGetLastError());
    c->n_trips = n;
    c->loaded = true;
    if (!scen) c->scen_trip_off = {0, n};
    TRY(reset_state(c));  // synchronises: the host vectors above may go away
    return LPSIM_OK;
}

// span slots for a chunk of c->C steps (kernel timing); the accumulators
// keep their sums
int timing_buffers(lpsim_ctx *c) {
    if (!c->d.tacc) {
        TRY(dnew(c, c->d.tacc, 16));
        CU(cudaMemsetAsync(c->d.tacc, 0, 16 * 8, c->stream));
    }
    if (c->tspan_steps < c->C) {
        TRY(dnew(c, c->tspan_buf, 2ull * (3ull * c->C + 1)));
        CU(cudaMemsetAsync(c->tspan_buf, 0, 2ull * (3ull * c->C + 1) * 8, c->stream));
        c->tspan_steps = c->C;
    }
    c->d.tspan = c->tspan_buf;
    c->d.tspan_light = 3 * c->C;
    CU(cudaStreamSynchronize(c->stream));
    return LPSIM_OK;
}

// launch configuration: block size, resident 256-thread blocks per SM, sort
// period and graph chunk; graphs are rebuilt on the next chunk
int apply_config(lpsim_ctx *c, uint32_t block, uint32_t bps, uint32_t R, uint32_t chunk) {
    CU(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < 2; i++)
        if (c->graph[i]) {
            cudaGraphExecDestroy(c->graph[i]);
            c->graph[i] = nullptr;
        }
    c->block = (int)block;
    c->grid = std::max(1, c->n_sm * (int)bps * 256 / (int)block);
    c->R = R;
    uint32_t base = 2 * R;
    base = base % 3 == 0 ? base : base * 3;
    c->C = std::max(base, (chunk + base - 1) / base * base);
    c->p.block_size = block;
    c->p.blocks_per_sm = bps;
    c->p.sort_period = R;
    c->p.chunk_steps = chunk;
    if (c->timing) TRY(timing_buffers(c));
    return LPSIM_OK;
}

int snapshot_impl(lpsim_ctx *c) {
    CU(cudaStreamSynchronize(c->stream));
    size_t total = 0;
    for (auto &b : c->mut) total += (b.second + 255) & ~size_t(255);
    if (!c->snap) {
        c->snap = static_cast<uint8_t *>(c->dalloc(total));
        if (!c->snap) return fail(LPSIM_E_OOM, "snapshot allocation failed");
        c->snap_bytes = total;
    }
    if (total != c->snap_bytes) return fail(LPSIM_E_STATE, "state layout changed since the first snapshot");
    size_t o = 0;
    for (auto &b : c->mut) {
        CU(cudaMemcpyAsync(c->snap + o, b.first, b.second, cudaMemcpyDeviceToDevice, c->stream));
        o += (b.second + 255) & ~size_t(255);
    }
    CU(cudaStreamSynchronize(c->stream));
    c->snap_host = {c->k, c->cur, c->stall_steps, c->last_progress};
    c->has_snap = true;
    return LPSIM_OK;
}

int restore_impl(lpsim_ctx *c) {
    if (!c->has_snap) return fail(LPSIM_E_STATE, "no snapshot taken");
    CU(cudaStreamSynchronize(c->stream));
    size_t o = 0;
    for (auto &b : c->mut) {
        CU(cudaMemcpyAsync(b.first, c->snap + o, b.second, cudaMemcpyDeviceToDevice, c->stream));
        o += (b.second + 255) & ~size_t(255);
    }
    CU(cudaStreamSynchronize(c->stream));
    c->k = c->snap_host.k;
    c->cur = c->snap_host.cur;
    c->stall_steps = c->snap_host.stall_steps;
    c->last_progress = c->snap_host.last_progress;
    return LPSIM_OK;
}

}  // namespace

extern "C" {

int lpsim_load_demand(lpsim_ctx *c, uint64_t n, const uint32_t *depart_step, const uint64_t *route_off,
                      const uint32_t *route_edges, uint32_t *out_vid) {
    if (c && c->scen_edge_off.size() > 2)
        return fail(LPSIM_E_STATE, "a batched context takes lpsim_load_demand_batch");
    return load_demand_impl(c, n, depart_step, route_off, route_edges, out_vid, nullptr, 1, nullptr);
}

int lpsim_set_vehicle_types(lpsim_ctx *c, uint32_t n_types, const lpsim_vehicle_type *types) {
    if (!c || !types) return fail(LPSIM_E_INVALID_ARG, "NULL argument");
    if (c->loaded) return fail(LPSIM_E_STATE, "vehicle types are set before the trips are loaded");
    if (n_types == 0 || n_types > LPSIM_MAX_VEHICLE_TYPES)
        return fail(LPSIM_E_INVALID_ARG, "n_types must be 1.." + std::to_string(LPSIM_MAX_VEHICLE_TYPES));
    for (uint32_t t = 0; t < n_types; t++) {
        const lpsim_vehicle_type &y = types[t];
        if (!(y.a > 0.0f) || !(y.b > 0.0f) || !(y.s0 >= 0.0f) || !std::isfinite(y.T) || !(y.vmax > 0.0f) ||
            !(y.vmax <= 254.0f))
            return fail(LPSIM_E_INVALID_ARG, "vehicle type " + std::to_string(t) + ": parameter out of range");
    }
    c->types.assign(types, types + n_types);
    return LPSIM_OK;
}

int lpsim_load_demand_typed(lpsim_ctx *c, uint64_t n, const uint32_t *depart_step, const uint64_t *route_off,
                            const uint32_t *route_edges, const uint8_t *vtype, uint32_t *out_vid) {
    if (c && c->scen_edge_off.size() > 2)
        return fail(LPSIM_E_STATE, "a batched context takes lpsim_load_demand_batch");
    return load_demand_impl(c, n, depart_step, route_off, route_edges, out_vid, nullptr, 1, nullptr, vtype);
}

int lpsim_load_demand_batch(lpsim_ctx *c, uint32_t n_scen, const uint64_t *n_trips, const uint32_t *const *depart_step,
                            const uint64_t *const *route_off, const uint32_t *const *route_edges,
                            const uint64_t *seeds, uint32_t *out_vid) {
    if (!c) return fail(LPSIM_E_INVALID_ARG, "ctx is NULL");
    if (n_scen == 0 || !n_trips || !depart_step || !route_off || !route_edges)
        return fail(LPSIM_E_INVALID_ARG, "batch array is NULL");
    if (c->scen_edge_off.size() != (size_t)n_scen + 1)
        return fail(LPSIM_E_INVALID_ARG, "n_scen does not match the batched network");
    uint64_t n = 0, tot = 0;
    for (uint32_t sc = 0; sc < n_scen; sc++) {
        if (!depart_step[sc] || !route_off[sc] || !route_edges[sc])
            return fail(LPSIM_E_INVALID_ARG, "scenario " + std::to_string(sc) + ": trip array is NULL");
        if (route_off[sc][0] != 0) return fail(LPSIM_E_INVALID_ARG, "route_off must start at 0");
        n += n_trips[sc];
        tot += route_off[sc][n_trips[sc]];
    }
    std::vector<uint32_t> dep(n), scen(n), edges(tot ? tot : 1);
    std::vector<uint64_t> off(n + 1);
    uint64_t j = 0, q = 0;
    off[0] = 0;
    c->scen_trip_off.assign(1, 0);
    for (uint32_t sc = 0; sc < n_scen; sc++) {
        const uint64_t eo = c->scen_edge_off[sc], ecount = c->scen_edge_off[sc + 1] - eo;
        for (uint64_t t = 0; t < n_trips[sc]; t++, j++) {
            dep[j] = depart_step[sc][t];
            scen[j] = sc;
            for (uint64_t r = route_off[sc][t]; r < route_off[sc][t + 1]; r++) {
                if (route_edges[sc][r] >= ecount)
                    return fail(LPSIM_E_INVALID_ARG, "scenario " + std::to_string(sc) + ": edge id out of range");
                edges[q++] = (uint32_t)(route_edges[sc][r] + eo);
            }
            off[j + 1] = q;
        }
        c->scen_trip_off.push_back(j);
    }
    return load_demand_impl(c, n, dep.data(), off.data(), edges.data(), out_vid, scen.data(), n_scen, seeds);
}

int lpsim_step(lpsim_ctx *c, uint32_t n_steps) {
    if (!c) return fail(LPSIM_E_INVALID_ARG, "ctx is NULL");
    if (!c->loaded) return fail(LPSIM_E_STATE, "lpsim_load_demand has not been called");
    uint64_t taken = 0;
    TRY(run_steps(c, n_steps, false, &taken));
    return read_status(c);
}

int lpsim_run(lpsim_ctx *c, uint32_t max_steps, lpsim_run_result *out) {
    if (!c) return fail(LPSIM_E_INVALID_ARG, "ctx is NULL");
    if (!c->loaded) return fail(LPSIM_E_STATE, "lpsim_load_demand has not been called");
    auto t0 = std::chrono::steady_clock::now();
    TRY(read_status(c));
    unsigned long long vs0 = c->h_ctr[0];
    uint64_t taken = 0;
    TRY(run_steps(c, max_steps, true, &taken));
    TRY(read_status(c));
    auto t1 = std::chrono::steady_clock::now();
    if (out) {
        out->steps = taken;
        out->veh_steps = c->h_ctr[0] - vs0;
        out->arrived = c->h_ctr[1];
        out->active = c->h_ctr[4] - c->h_ctr[1];
        out->waiting = c->n_trips - c->h_ctr[4];
        out->k = c->k;
        out->wall_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    }
    return LPSIM_OK;
}

int lpsim_reset(lpsim_ctx *c) {
    if (!c) return fail(LPSIM_E_INVALID_ARG, "ctx is NULL");
    return reset_state(c);
}

int lpsim_link_stats(lpsim_ctx *c, lpsim_link_stat *out, uint64_t n_edges, uint32_t *bin_inflow, uint32_t *bin_tt_sum,
                     uint32_t *bin_tt_cnt, uint32_t *bin_occ, uint32_t n_bins) {
    if (!c) return fail(LPSIM_E_INVALID_ARG, "ctx is NULL");
    if (n_edges != c->n_edges) return fail(LPSIM_E_INVALID_ARG, "n_edges does not match the network");
    if ((bin_inflow || bin_tt_sum || bin_tt_cnt || bin_occ) && n_bins != c->p.n_bins)
        return fail(LPSIM_E_INVALID_ARG, "n_bins does not match the context");
    CU(cudaStreamSynchronize(c->stream));
    if (out) {
        std::vector<unsigned long long> a(c->n_edges), b(c->n_edges), t(c->n_edges);
        CU(cudaMemcpy(a.data(), c->d.ent, c->n_edges * 8ull, cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(b.data(), c->d.ext, c->n_edges * 8ull, cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(t.data(), c->d.tts, c->n_edges * 8ull, cudaMemcpyDeviceToHost));
        for (uint32_t e = 0; e < c->n_edges; e++) out[e] = lpsim_link_stat{a[e], b[e], t[e]};
    }
    size_t nb = (size_t)c->n_edges * c->p.n_bins * 4;
    if (nb) {
        // device arrays are bin-major: transpose into edge-major scratch first
        Scratch scratch(c, nb);
        if (!scratch.p) return fail(LPSIM_E_OOM, "device scratch allocation failed");
        uint32_t *tmp = static_cast<uint32_t *>(scratch.p);
        struct {
            uint32_t *host;
            const uint32_t *dev;
        } outs[] = {{bin_inflow, c->d.bin_in}, {bin_tt_sum, c->d.bin_tt}, {bin_tt_cnt, c->d.bin_cnt},
                    {bin_occ, c->d.bin_occ}};
        int rc = LPSIM_OK;
        for (auto &o : outs) {
            if (!o.host) continue;
            launch_transpose_bins(o.dev, c->n_edges, c->p.n_bins, tmp, c->stream);
            cudaError_t e = cudaMemcpyAsync(o.host, tmp, nb, cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) {
                rc = fail(LPSIM_E_CUDA, std::string("link statistics: ") + cudaGetErrorString(e));
                break;
            }
        }
        if (rc) return rc;
    }
    return LPSIM_OK;
}

int lpsim_get_trips(lpsim_ctx *c, uint64_t n, uint32_t *depart_actual, uint32_t *arrive_step) {
    if (!c) return fail(LPSIM_E_INVALID_ARG, "ctx is NULL");
    if (!c->loaded) return fail(LPSIM_E_STATE, "lpsim_load_demand has not been called");
    if (n != c->n_trips) return fail(LPSIM_E_INVALID_ARG, "n does not match the trips loaded");
    CU(cudaStreamSynchronize(c->stream));
    if (depart_actual) CU(cudaMemcpy(depart_actual, c->d.dep_act, n * 4, cudaMemcpyDeviceToHost));
    if (arrive_step) CU(cudaMemcpy(arrive_step, c->d.arr, n * 4, cudaMemcpyDeviceToHost));
    return LPSIM_OK;
}

int lpsim_get_state(lpsim_ctx *c, uint64_t n, float *x, float *v, uint32_t *edge, uint8_t *lane, uint32_t *ridx,
                    uint8_t *status) {
    if (!c) return fail(LPSIM_E_INVALID_ARG, "ctx is NULL");
    if (!c->loaded) return fail(LPSIM_E_STATE, "lpsim_load_demand has not been called");
    if (n != c->n_trips) return fail(LPSIM_E_INVALID_ARG, "n does not match the trips loaded");
    // scratch: x, v, edge, ridx (4 B each) and lane (1 B) per vehicle; given
    // back on every exit path (after the stream has finished with it)
    Scratch scratch(c, n * 17 + 64);
    if (!scratch.p) return fail(LPSIM_E_OOM, "device scratch allocation failed");
    uint8_t *tmp = static_cast<uint8_t *>(scratch.p);
    float *dx = reinterpret_cast<float *>(tmp);
    float *dv = dx + n;
    uint32_t *de = reinterpret_cast<uint32_t *>(dv + n);
    uint32_t *dr = de + n;
    uint8_t *dl = reinterpret_cast<uint8_t *>(dr + n);
    CU(cudaMemsetAsync(tmp, 0, n * 17, c->stream));
    CU(cudaMemsetAsync(de, 0xFF, n * 4, c->stream));
    Dev d = c->d;
    d.s = c->sets[c->cur];
    launch_state_scatter(d, c->k, dx, dv, de, dl, dr, c->stream);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(c->stream));
    if (x) CU(cudaMemcpy(x, dx, n * 4, cudaMemcpyDeviceToHost));
    if (v) CU(cudaMemcpy(v, dv, n * 4, cudaMemcpyDeviceToHost));
    if (edge) CU(cudaMemcpy(edge, de, n * 4, cudaMemcpyDeviceToHost));
    if (ridx) CU(cudaMemcpy(ridx, dr, n * 4, cudaMemcpyDeviceToHost));
    if (lane) CU(cudaMemcpy(lane, dl, n, cudaMemcpyDeviceToHost));
    if (status) CU(cudaMemcpy(status, c->d.status, n, cudaMemcpyDeviceToHost));
    return LPSIM_OK;
}

uint64_t lpsim_lane_map_size(const lpsim_ctx *c) { return c ? c->canon_cells : 0; }

int lpsim_get_lane_map(lpsim_ctx *c, uint8_t *out, uint64_t size) {
    if (!c || !out) return fail(LPSIM_E_INVALID_ARG, "NULL argument");
    if (size != c->canon_cells) return fail(LPSIM_E_INVALID_ARG, "size must equal lpsim_lane_map_size()");
    CU(cudaStreamSynchronize(c->stream));
    std::vector<uint8_t> m(c->map_bytes);
    CU(cudaMemcpy(m.data(), c->d.map[c->k % 3], c->map_bytes, cudaMemcpyDeviceToHost));
    uint64_t o = 0;
    for (uint32_t e = 0; e < c->n_edges; e++) {
        uint32_t stride = row_stride(c->len[e]);
        for (uint32_t l = 0; l < c->lanes[e]; l++) {
            std::memcpy(out + o, m.data() + c->moff[e] + (uint64_t)l * stride, c->len[e]);
            o += c->len[e];
        }
    }
    return LPSIM_OK;
}

int lpsim_get_counters(lpsim_ctx *c, lpsim_counters *out) {
    if (!c || !out) return fail(LPSIM_E_INVALID_ARG, "NULL argument");
    TRY(read_status(c));
    out->k = c->k;
    out->veh_steps = c->h_ctr[0];
    out->arrived = c->h_ctr[1];
    out->active = c->h_ctr[4] - c->h_ctr[1];
    out->waiting = c->n_trips - c->h_ctr[4];
    out->lane_changes = c->h_ctr[2];
    out->slots = c->h_ctr[9] & 0xFFFFFFFFull;
    out->launches = c->launches;
    out->light_chunks = c->light_chunks;
    return LPSIM_OK;
}

int lpsim_set_kernel_timing(lpsim_ctx *c, int on) {
    if (!c) return fail(LPSIM_E_INVALID_ARG, "ctx is NULL");
    CU(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < 2; i++)
        if (c->graph[i]) {
            cudaGraphExecDestroy(c->graph[i]);
            c->graph[i] = nullptr;
        }
    if (on) {
        TRY(timing_buffers(c));
        CU(cudaMemsetAsync(c->d.tacc, 0, 16 * 8, c->stream));
        CU(cudaStreamSynchronize(c->stream));
        c->timing = true;
    } else {
        // the sums stay readable; the kernels stop stamping
        c->timing = false;
        c->d.tspan = nullptr;
    }
    return LPSIM_OK;
}

int lpsim_get_kernel_times(lpsim_ctx *c, lpsim_kernel_times *out) {
    if (!c || !out) return fail(LPSIM_E_INVALID_ARG, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    if (!c->d.tacc) return LPSIM_OK;
    unsigned long long a[16];
    CU(cudaStreamSynchronize(c->stream));
    CU(cudaMemcpy(a, c->d.tacc, sizeof(a), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 4; i++) {
        out->ms[i] = (double)a[i] * 1e-6;
        out->launches[i] = a[4 + i];
    }
    out->p1_veh_steps = a[8];
    return LPSIM_OK;
}

int lpsim_snapshot(lpsim_ctx *c) {
    if (!c) return fail(LPSIM_E_INVALID_ARG, "ctx is NULL");
    if (!c->loaded) return fail(LPSIM_E_STATE, "lpsim_load_demand has not been called");
    return snapshot_impl(c);
}

int lpsim_restore(lpsim_ctx *c) {
    if (!c) return fail(LPSIM_E_INVALID_ARG, "ctx is NULL");
    return restore_impl(c);
}

int lpsim_autotune(lpsim_ctx *c, uint32_t window_steps, lpsim_tune_result *out) {
    if (!c) return fail(LPSIM_E_INVALID_ARG, "ctx is NULL");
    if (!c->loaded) return fail(LPSIM_E_STATE, "lpsim_load_demand has not been called");
    if (window_steps == 0) return fail(LPSIM_E_INVALID_ARG, "window_steps must be > 0");
    const uint32_t cur_cfg[4] = {(uint32_t)c->block, c->p.blocks_per_sm ? c->p.blocks_per_sm : 4u, c->R,
                                 c->p.chunk_steps ? c->p.chunk_steps : 1536u};
    TRY(snapshot_impl(c));
    // candidates run without kernel timing
    const bool timing = c->timing;
    c->timing = false;
    c->d.tspan = nullptr;
    struct Cand {
        uint32_t block, bps, R;
    };
    std::vector<Cand> cands;
    cands.push_back({cur_cfg[0], cur_cfg[1], cur_cfg[2]});
    for (uint32_t R : {64u, 128u, 256u})
        for (uint32_t block : {128u, 256u, 512u})
            for (uint32_t bps : {2u, 4u, 6u})
                if (!(block == cur_cfg[0] && bps == cur_cfg[1] && R == cur_cfg[2])) cands.push_back({block, bps, R});
    double best = 1e300, dflt = 0.0;
    Cand pick = cands[0];
    for (size_t i = 0; i < cands.size(); i++) {
        const Cand &cd = cands[i];
        TRY(apply_config(c, cd.block, cd.bps, cd.R, cur_cfg[3]));
        TRY(restore_impl(c));
        // capture the graphs outside the timed window
        if (c->k % c->C == 0) TRY(capture_chunk(c, c->cur));
        uint64_t taken = 0;
        auto t0 = std::chrono::steady_clock::now();
        TRY(run_steps(c, window_steps, false, &taken));
        auto t1 = std::chrono::steady_clock::now();
        double ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
        if (i == 0) dflt = ms;
        if (ms < best) {
            best = ms;
            pick = cd;
        }
    }
    TRY(apply_config(c, pick.block, pick.bps, pick.R, cur_cfg[3]));
    TRY(restore_impl(c));
    if (timing) {
        c->timing = true;
        TRY(timing_buffers(c));
    }
    if (out) {
        out->block_size = pick.block;
        out->blocks_per_sm = pick.bps;
        out->sort_period = pick.R;
        out->chunk_steps = c->C;
        out->best_ms = best;
        out->default_ms = dflt;
        out->n_tried = (uint32_t)cands.size();
    }
    return LPSIM_OK;
}

int lpsim_set_config(lpsim_ctx *c, uint32_t block_size, uint32_t blocks_per_sm, uint32_t sort_period,
                     uint32_t chunk_steps) {
    if (!c) return fail(LPSIM_E_INVALID_ARG, "ctx is NULL");
    if (block_size != 128 && block_size != 256 && block_size != 512)
        return fail(LPSIM_E_INVALID_ARG, "block_size must be 128, 256 or 512");
    if (blocks_per_sm == 0 || blocks_per_sm > 8 || sort_period == 0 || sort_period > 256 || chunk_steps == 0)
        return fail(LPSIM_E_INVALID_ARG, "configuration value out of range");
    return apply_config(c, block_size, blocks_per_sm, sort_period, chunk_steps);
}

void lpsim_destroy(lpsim_ctx *c) { delete c; }

}  // extern "C"
