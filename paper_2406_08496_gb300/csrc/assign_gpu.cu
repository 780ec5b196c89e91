// Time-dependent shortest paths of the assignment loop on the GPU.
//
// The assignment loop (method of successive averages around the simulator)
// needs, every iteration, the earliest-arrival path of every trip under the
// link times of that iteration: routing is the step upstream of the
// simulation ("after the routing", Sec. 3.1), and re-routing between
// simulations is the paper's stated next step (Sec. 5).  Trips with the same
// origin and 30-minute departure period share one tree rooted at the middle
// of the period; at the regional scale that is some 10^5 trees per iteration
// on a 224k-node graph, far more than the host's threads finish in seconds.
//
// Here every tree is searched by one warp, thousands of warps at a time (a
// tree's frontier is a wave of a few hundred nodes; many trees in flight
// hide the memory latency each relaxation pays: on the 2.82M-trip day, 16
// trees per SM took 2.7 s per pass, 32 took 1.85 s, 64 took 1.78 s; the
// out-edges of a round's near nodes spread over the lanes took 32 to 1.7 s,
// a node's label, round stamp and far mark in one 16-byte record to
// 1.33 s, and 40 trees per SM (48 registers, no spills) to 1.26 s):
//   * label-correcting search in rounds over time buckets (near-far): the
//     near set's nodes relax their out-edges with the arrival function of
//     the bin holding their arrival time (FIFO by construction, see TD); a
//     node whose label improved joins the next round's near set when its
//     arrival is below the bucket threshold (once per round: a round stamp)
//     and the far pile otherwise (once: a mark); when the near set empties,
//     every label below the threshold is final, the threshold moves on by
//     the bucket width and the far nodes below it become the near set --
//     close to Dijkstra's work, with a whole near set relaxed per round;
//   * a label is (arrival ms << 32 | entering edge id) in one 64-bit word,
//     so atomicMin keeps the earliest arrival and, among equal arrivals, the
//     lower edge id -- the fixed point is exactly the tree the host's
//     Dijkstra builds (lpsim_assign_shortest_paths), with integer millisecond
//     link times making every arrival an exact sum;
//   * the search ends once every destination of the group is below the
//     threshold (settled); until then the latest destination label bounds
//     it: a node reached later cannot lie on any of their paths (link times
//     are positive), so it is not expanded;
//   * each trip's path is read back along the entering edges, written to the
//     output in travel order and timed from the trip's own departure;
//   * the labels the tree set are reset from its list of reached nodes, so a
//     warp's workspace is reused without clearing the whole graph.
// Every loop is bounded (rounds and path walks by the node count); a bound
// that is hit sets an error bit the host reports.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "../../include/lpsim_assign.h"
#include "assign_internal.h"
#include "host_par.h"

int lpsim_fail(int code, const std::string &msg);

using namespace lpsim_assign_detail;

namespace {

int fail(int code, const std::string &m) { return lpsim_fail(code, m); }

#define CU(call)                                                                                      \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return fail(LPSIM_E_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

constexpr uint64_t kUnreached = ~0ull;
constexpr uint32_t kNoEdge = 0xFFFFFFFFu;
#ifndef LPSIM_ASSIGN_WARPS_PER_SM
#define LPSIM_ASSIGN_WARPS_PER_SM 40
#endif
#ifndef LPSIM_ASSIGN_WORKSPACE_GIB
#define LPSIM_ASSIGN_WORKSPACE_GIB 48
#endif
constexpr int kWarpsPerBlock = 4;
constexpr int kBlocksPerSm = LPSIM_ASSIGN_WARPS_PER_SM / kWarpsPerBlock;   // trees searched at once per SM / 4
constexpr uint64_t kWorkspaceBudget = (uint64_t)LPSIM_ASSIGN_WORKSPACE_GIB << 30;  // per-warp workspaces at most
#ifndef LPSIM_ASSIGN_DELTA_MS
#define LPSIM_ASSIGN_DELTA_MS 60000
#endif
constexpr uint64_t kDeltaMs = LPSIM_ASSIGN_DELTA_MS;  // bucket width of the search thresholds (ms)

// error bits
constexpr uint32_t kErrUnreachable = 1u;  // a destination not reached (or equal to its origin)
constexpr uint32_t kErrCapacity = 2u;     // the path buffer was too small (the host retries)
constexpr uint32_t kErrBound = 4u;        // a round or path-walk bound was hit

struct GroupRec {
    uint32_t src;    // origin node
    uint32_t t0;     // root time (ms)
    uint32_t first;  // first position in the trip order
    uint32_t count;  // trips
};

// a node's search state in one 16-byte record, so the atomics of one
// relaxation (the label's minimum, then the round stamp or the far mark)
// touch one 32-byte sector
struct __align__(16) NodeRec {
    unsigned long long lab;  // (arrival ms << 32) | entering edge, or all ones while unreached
    uint32_t inq;            // round stamp of the last push onto a near set
    uint32_t fmark;          // tree mark while the node is in the far pile
};

struct TreeArgs {
    uint32_t n_nodes, n_edges, n_bins, bin_ms;
    const uint32_t *out_off;  // n_nodes + 1
    const uint2 *adj;         // per out-edge position: {edge, head node}
    const uint32_t *src;      // per edge: tail node
    const uint2 *cms;         // n_bins x n_edges: {link time ms, earliest arrival entering a later bin ms}
    uint32_t n_groups;
    const GroupRec *groups;
    const uint32_t *order;    // trip per position, group by group
    const uint32_t *dest;     // per trip
    const uint32_t *dep_ms;   // per trip: planned departure (ms)
    // outputs per trip
    unsigned long long *path_off;
    uint32_t *path_len;
    float *tsp;
    uint32_t *edges;          // path edges, travel order
    unsigned long long cap;   // entries of edges
    unsigned long long *cursor;
    // per-warp workspaces
    NodeRec *node;            // n_warps x n_nodes: label, round stamp of the last push, far-pile mark
    uint32_t *touched;        // n_warps x n_nodes
    uint32_t *fa, *fb;        // n_warps x n_nodes: near sets (this round, next round)
    uint32_t *far;            // n_warps x n_nodes: far pile (labels at or above the threshold)
    uint32_t *stamp;          // per warp: last round stamp used
    uint64_t delta_ms;        // bucket width of the thresholds
    uint32_t *next_group;
    uint32_t *err;
};

__device__ __forceinline__ uint32_t bin_of(const TreeArgs &A, uint64_t t) {
    const uint64_t b = t / A.bin_ms;
    return b < A.n_bins ? (uint32_t)b : A.n_bins - 1u;
}

// arrival when entering edge e at time t (ms): min(t + c, M) of t's bin
__device__ __forceinline__ uint64_t arrive(const uint2 lt, uint64_t t) {
    const uint64_t a = t + lt.x;
    return a < (uint64_t)lt.y ? a : (uint64_t)lt.y;
}

// Latest current arrival over the group's destinations (its trips'), or
// kUnreached while any is unreached; every lane gets the result.
__device__ __forceinline__ uint64_t dest_bound(const TreeArgs &A, const GroupRec &G, const NodeRec *nd,
                                               uint32_t lane) {
    uint64_t m = 0;
    for (uint32_t q = lane; q < G.count; q += 32) {
        const uint64_t l = __ldcg(&nd[A.dest[A.order[G.first + q]]].lab);
        const uint64_t t = l == kUnreached ? kUnreached : (l >> 32);
        m = t > m ? t : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t y = __shfl_xor_sync(0xFFFFFFFFu, m, o);
        m = y > m ? y : m;
    }
    return m;
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32, kBlocksPerSm) td_trees(TreeArgs A) {
    const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    const size_t gw = (size_t)blockIdx.x * kWarpsPerBlock + wib;
    NodeRec *nd = A.node + gw * A.n_nodes;
    uint32_t *touched = A.touched + gw * A.n_nodes;
    uint32_t *fa = A.fa + gw * A.n_nodes, *fb = A.fb + gw * A.n_nodes;
    uint32_t *far = A.far + gw * A.n_nodes;
    __shared__ uint32_t s_next[kWarpsPerBlock], s_touched[kWarpsPerBlock], s_far[kWarpsPerBlock];
    uint32_t stamp = A.stamp[gw];
    // rounds of a search at most: every round settles or re-labels a node,
    // and a node's label improves a bounded number of times
    const uint64_t max_rounds = 8ull * A.n_nodes + (1ull << 20);
    for (;;) {
        uint32_t g = 0;
        if (lane == 0) g = atomicAdd(A.next_group, 1u);
        g = __shfl_sync(0xFFFFFFFFu, g, 0);
        if (g >= A.n_groups) break;
        const GroupRec G = A.groups[g];
        const uint32_t tmark = ++stamp;  // this tree's mark of the nodes in its far pile
        if (lane == 0) {
            __stcg(&nd[G.src].lab, (unsigned long long)(((uint64_t)G.t0 << 32) | kNoEdge));
            __stcg(touched, G.src);
            __stcg(fa, G.src);
        }
        uint32_t nn = 1, nt = 1, nfar = 0;
        uint64_t theta = (uint64_t)G.t0 + A.delta_ms;  // labels below theta are expanded now, the rest wait
        uint64_t ub = kUnreached;  // latest destination arrival so far (ms), once all are reached
        __threadfence_block();
        __syncwarp();
        bool bounded = true;
        for (uint64_t round = 0;; round++) {
            if (round > max_rounds) {
                bounded = false;
                break;
            }
            if (nn > 0) {
                // one round of the near set: relax the out-edges of its nodes
                stamp++;
                if (lane == 0) {
                    s_next[wib] = 0;
                    s_touched[wib] = nt;
                    s_far[wib] = nfar;
                }
                __syncwarp();
                // 32 near nodes at a time, their out-edges spread over the
                // lanes (a warp scan of the degrees; each lane finds the node
                // of its edge by a binary search over the scan), so a round
                // with a few nodes of a few edges each keeps most lanes busy
                for (uint32_t c0 = 0; c0 < nn; c0 += 32) {
                    const uint32_t i = c0 + lane;
                    uint32_t u = 0, j0 = 0, deg = 0;
                    uint64_t tu = kUnreached;
                    if (i < nn) {
                        u = __ldcg(fa + i);
                        tu = __ldcg(&nd[u].lab) >> 32;
                        j0 = A.out_off[u];
                        deg = tu < ub ? A.out_off[u + 1] - j0 : 0u;
                    }
                    uint32_t incl = deg;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                        if (lane >= (uint32_t)o) incl += y;
                    }
                    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
                    for (uint32_t b0 = 0; b0 < total; b0 += 32) {
                        const uint32_t t = b0 + lane;
                        // the lane whose node owns edge t: the first with incl > t
                        uint32_t owner = 0;
#pragma unroll
                        for (uint32_t step = 16; step > 0; step >>= 1) {
                            const uint32_t y = __shfl_sync(0xFFFFFFFFu, incl, (int)(owner + step - 1));
                            if (y <= t) owner += step;
                        }
                        const uint32_t o_incl = __shfl_sync(0xFFFFFFFFu, incl, (int)owner);
                        const uint32_t o_deg = __shfl_sync(0xFFFFFFFFu, deg, (int)owner);
                        const uint32_t o_j0 = __shfl_sync(0xFFFFFFFFu, j0, (int)owner);
                        const uint64_t o_tu = __shfl_sync(0xFFFFFFFFu, tu, (int)owner);
                        if (t >= total) continue;
                        const uint32_t j = o_j0 + (t - (o_incl - o_deg));
                        const uint2 ev = A.adj[j];
                        const uint64_t at = arrive(A.cms[(size_t)bin_of(A, o_tu) * A.n_edges + ev.x], o_tu);
                        if (at > 0xFFFFFFFFull || at > ub) continue;
                        const unsigned long long cand = (at << 32) | ev.x;
                        const unsigned long long old = atomicMin(&nd[ev.y].lab, cand);
                        if (cand < old) {
                            if (old == kUnreached) __stcg(touched + atomicAdd(&s_touched[wib], 1u), ev.y);
                            if (at < theta) {
                                if (atomicExch(&nd[ev.y].inq, stamp) != stamp)
                                    __stcg(fb + atomicAdd(&s_next[wib], 1u), ev.y);
                            } else if (atomicExch(&nd[ev.y].fmark, tmark) != tmark) {
                                __stcg(far + atomicAdd(&s_far[wib], 1u), ev.y);
                            }
                        }
                    }
                }
                __threadfence_block();
                __syncwarp();
                nn = s_next[wib];
                nt = s_touched[wib];
                nfar = s_far[wib];
                uint32_t *t = fa;
                fa = fb;
                fb = t;
                __syncwarp();
                continue;
            }
            // the near set is empty: every label below theta is final
            ub = dest_bound(A, G, nd, lane);
            if (ub < theta || nfar == 0) break;  // every destination settled (or nothing left)
            // next threshold: move the far nodes below it to the near set, keep
            // the rest (the far list holds each node once: its mark)
            uint64_t next = theta + A.delta_ms;
            for (int pass = 0; pass < 2 && nn == 0 && nfar > 0; pass++) {
                uint32_t kept = 0;
                uint64_t tmin = kUnreached;
                for (uint32_t c0 = 0; c0 < nfar; c0 += 32) {
                    const uint32_t i = c0 + lane;
                    uint32_t v = 0;
                    uint64_t tv = kUnreached;
                    if (i < nfar) {
                        v = __ldcg(far + i);
                        tv = __ldcg(&nd[v].lab) >> 32;
                    }
                    const bool drop = i < nfar && tv < theta;            // settled in an earlier bucket
                    const bool move = i < nfar && tv >= theta && tv < next;
                    const bool keep = i < nfar && tv >= next;
                    const uint32_t mk = __ballot_sync(0xFFFFFFFFu, keep), mm = __ballot_sync(0xFFFFFFFFu, move);
                    const uint32_t below = (1u << lane) - 1u;
                    __syncwarp();  // every lane has read its entry before any is overwritten
                    if (drop || move) __stcg(&nd[v].fmark, 0u);
                    if (keep) __stcg(far + kept + __popc(mk & below), v);
                    if (move) __stcg(fa + nn + __popc(mm & below), v);
                    kept += __popc(mk);
                    nn += __popc(mm);
                    uint64_t tk = keep ? tv : kUnreached;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const uint64_t y = __shfl_xor_sync(0xFFFFFFFFu, tk, o);
                        tk = y < tk ? y : tk;
                    }
                    tmin = tk < tmin ? tk : tmin;
                }
                nfar = kept;
                theta = next;
                // nothing below the threshold: jump to the earliest far label
                if (nn == 0 && nfar > 0) next = tmin + A.delta_ms;
            }
            __threadfence_block();
            __syncwarp();
        }
        if (!bounded && lane == 0) atomicOr(A.err, kErrBound);
        // far marks of the nodes still in the far pile (the others were cleared)
        for (uint32_t i = lane; i < nfar; i += 32) __stcg(&nd[__ldcg(far + i)].fmark, 0u);
        // paths of the group's trips, in travel order, timed from each trip's departure
        for (uint32_t q = lane; q < G.count; q += 32) {
            const uint32_t j = A.order[G.first + q];
            const uint32_t d = A.dest[j];
            A.path_len[j] = 0;
            const uint64_t ld = __ldcg(&nd[d].lab);
            if (ld == kUnreached || d == G.src || !bounded) {
                atomicOr(A.err, kErrUnreachable);
                continue;
            }
            uint32_t L = 0;
            bool ok = true;
            for (uint32_t v = d; v != G.src;) {
                const uint32_t e = (uint32_t)__ldcg(&nd[v].lab);
                if (++L > A.n_nodes || e >= A.n_edges) {
                    ok = false;
                    break;
                }
                v = A.src[e];
            }
            if (!ok) {
                atomicOr(A.err, kErrBound);
                continue;
            }
            const unsigned long long off = atomicAdd(A.cursor, (unsigned long long)L);
            if (off + L > A.cap) {
                atomicOr(A.err, kErrCapacity);
                continue;
            }
            uint32_t pos = L;
            for (uint32_t v = d; v != G.src && pos > 0;) {
                const uint32_t e = (uint32_t)__ldcg(&nd[v].lab);
                A.edges[off + --pos] = e;  // e < n_edges: the counting walk checked this chain
                v = A.src[e];
            }
            const uint64_t tj = A.dep_ms[j];
            uint64_t t = tj;
            for (uint32_t p = 0; p < L; p++) t = arrive(A.cms[(size_t)bin_of(A, t) * A.n_edges + A.edges[off + p]], t);
            A.path_off[j] = off;
            A.path_len[j] = L;
            A.tsp[j] = (float)((double)(t - tj) / 1000.0);
        }
        // clear the labels this tree set
        __syncwarp();
        for (uint32_t i = lane; i < nt; i += 32)
            __stcg(&nd[__ldcg(touched + i)].lab, (unsigned long long)kUnreached);
        __threadfence_block();
        __syncwarp();
    }
    if (lane == 0) A.stamp[gw] = stamp;
}

// every node unreached, with no round stamp and no far mark
__global__ void init_nodes(NodeRec *nd, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        nd[i] = NodeRec{(unsigned long long)kUnreached, 0u, 0u};
}

// Inflow per (edge, bin) of the routes: each trip walks its route from its
// planned departure with the arrival rule of the table, counting one entry
// in the bin of every link entry time (the host's lpsim_assign_load, on the
// device: integer counts, so the order of the atomics does not matter).
__global__ void load_routes(const unsigned long long *roff, const uint32_t *redge, const uint32_t *dep_ms,
                            uint64_t n, const uint2 *cms, uint32_t n_edges, uint32_t n_bins, uint32_t bin_ms,
                            uint32_t *inflow) {
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t t = dep_ms[j];
        const unsigned long long q1 = roff[j + 1];
        for (unsigned long long q = roff[j]; q < q1; q++) {
            const uint32_t e = redge[q];
            const uint64_t b = t / bin_ms;
            if (b < n_bins) atomicAdd(&inflow[(size_t)e * n_bins + b], 1u);
            t = arrive(cms[(size_t)(b < n_bins ? b : n_bins - 1) * n_edges + e], t);
        }
    }
}

}  // namespace

// Device copy of the graph, the trip table and the search workspaces.
struct AssignGpu {
    int device = -1;
    int n_sm = 0;
    cudaStream_t stream = nullptr;
    std::vector<void *> blocks;
    uint32_t n_warps = 0;
    TreeArgs A{};
    uint32_t period_steps = 0;  // grouping held in A.groups / A.order
    std::vector<uint64_t> order, gstart;
    unsigned long long cap = 0;
    // routes and inflow of lpsim_assign_load_gpu
    unsigned long long *roff = nullptr;
    uint32_t *redge = nullptr;
    uint64_t redge_cap = 0;
    uint32_t *inflow = nullptr;
    size_t inflow_cells = 0;
    // host staging kept between calls (grown, never shrunk, never cleared:
    // every call writes what it reads), so the large tables are not
    // zero-filled and their pages not faulted in again at every call
    std::unique_ptr<LinkTime[]> h_table;
    size_t h_table_cap = 0;
    std::unique_ptr<uint32_t[]> h_edges;
    size_t h_edges_cap = 0;
    LinkTime *table_buf(size_t n) {
        if (n > h_table_cap) {
            h_table.reset(new (std::nothrow) LinkTime[n]);
            h_table_cap = h_table ? n : 0;
        }
        return h_table.get();
    }
    uint32_t *edges_buf(size_t n) {
        n = std::max<size_t>(n, 1);
        if (n > h_edges_cap) {
            const size_t want = n + n / 4;
            h_edges.reset(new (std::nothrow) uint32_t[want]);
            h_edges_cap = h_edges ? want : 0;
        }
        return h_edges.get();
    }

    void *alloc(size_t bytes) {
        void *p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
        blocks.push_back(p);
        return p;
    }
    void release(void *p) {
        auto it = std::find(blocks.begin(), blocks.end(), p);
        if (it != blocks.end()) {
            blocks.erase(it);
            cudaFree(p);
        }
    }
    ~AssignGpu() {
        if (stream) cudaStreamSynchronize(stream);
        for (void *b : blocks) cudaFree(b);
        if (stream) cudaStreamDestroy(stream);
    }
};

void assign_gpu_free(AssignGpu *g) { delete g; }

namespace {

template <class T>
int dput(AssignGpu *g, T *&dst, const T *src, size_t count) {
    dst = static_cast<T *>(g->alloc(count * sizeof(T)));
    if (!dst) return fail(LPSIM_E_OOM, "device allocation of " + std::to_string(count * sizeof(T)) + " bytes failed");
    if (count) CU(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyHostToDevice, g->stream));
    return LPSIM_OK;
}

#define TRY(x)                           \
    do {                                 \
        int rc_ = (x);                   \
        if (rc_ != LPSIM_OK) return rc_; \
    } while (0)

// graph, trips and workspaces (first call)
int gpu_setup(lpsim_assign *a) {
    auto *g = new (std::nothrow) AssignGpu();
    if (!g) return fail(LPSIM_E_OOM, "host allocation failed");
    a->gpu = g;
    CU(cudaGetDevice(&g->device));
    CU(cudaDeviceGetAttribute(&g->n_sm, cudaDevAttrMultiProcessorCount, g->device));
    CU(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
    if (a->n >= 0xFFFFFFFFull) return fail(LPSIM_E_INVALID_ARG, "too many trips for the GPU search");
    TreeArgs &A = g->A;
    A.n_nodes = a->n_nodes;
    A.n_edges = a->n_edges;
    std::vector<uint2> adj(a->n_edges);
    for (uint32_t j = 0; j < a->n_edges; j++) adj[j] = make_uint2(a->out_edge[j], a->dst[a->out_edge[j]]);
    std::vector<uint32_t> dep_ms(a->n);
    for (uint64_t j = 0; j < a->n; j++) {
        const uint64_t t = to_ms((double)a->dep[j] * a->dt);
        if (t > 0xFFFFFFFFull) return fail(LPSIM_E_INVALID_ARG, "departure beyond the 32-bit millisecond range");
        dep_ms[j] = (uint32_t)t;
    }
    uint32_t *oo, *sr, *de, *dm;
    uint2 *ad;
    TRY(dput(g, oo, a->out_off.data(), a->out_off.size()));
    TRY(dput(g, ad, adj.data(), adj.size()));
    TRY(dput(g, sr, a->src.data(), a->src.size()));
    TRY(dput(g, de, a->dest.data(), a->dest.size()));
    TRY(dput(g, dm, dep_ms.data(), dep_ms.size()));
    A.out_off = oo;
    A.adj = ad;
    A.src = sr;
    A.dest = de;
    A.dep_ms = dm;
    A.path_off = static_cast<unsigned long long *>(g->alloc(a->n * 8));
    A.path_len = static_cast<uint32_t *>(g->alloc(a->n * 4));
    A.tsp = static_cast<float *>(g->alloc(a->n * 4));
    A.cursor = static_cast<unsigned long long *>(g->alloc(8));
    A.next_group = static_cast<uint32_t *>(g->alloc(4));
    A.err = static_cast<uint32_t *>(g->alloc(4));
    if (!A.path_off || !A.path_len || !A.tsp || !A.cursor || !A.next_group || !A.err)
        return fail(LPSIM_E_OOM, "device allocation failed");
    // workspaces: as many warps as fit the budget, at most kBlocksPerSm * kWarpsPerBlock per SM
    const uint64_t per_warp = (uint64_t)a->n_nodes * (sizeof(NodeRec) + 4 * 4);
    uint64_t warps = std::min<uint64_t>((uint64_t)g->n_sm * kBlocksPerSm * kWarpsPerBlock,
                                        std::max<uint64_t>(kWorkspaceBudget / std::max<uint64_t>(per_warp, 1), 1));
    warps = std::max<uint64_t>(kWarpsPerBlock, warps / kWarpsPerBlock * kWarpsPerBlock);
    g->n_warps = (uint32_t)warps;
    const size_t nn = (size_t)warps * a->n_nodes;
    A.node = static_cast<NodeRec *>(g->alloc(nn * sizeof(NodeRec)));
    A.touched = static_cast<uint32_t *>(g->alloc(nn * 4));
    A.fa = static_cast<uint32_t *>(g->alloc(nn * 4));
    A.fb = static_cast<uint32_t *>(g->alloc(nn * 4));
    A.far = static_cast<uint32_t *>(g->alloc(nn * 4));
    A.stamp = static_cast<uint32_t *>(g->alloc(warps * 4));
    if (!A.node || !A.touched || !A.fa || !A.fb || !A.far || !A.stamp)
        return fail(LPSIM_E_OOM, "device allocation of the search workspaces failed");
    init_nodes<<<g->n_sm * 4, 256, 0, g->stream>>>(A.node, nn);
    CU(cudaGetLastError());
    A.delta_ms = kDeltaMs;
    CU(cudaMemsetAsync(A.stamp, 0, warps * 4, g->stream));
    CU(cudaStreamSynchronize(g->stream));
    return LPSIM_OK;
}

// trip groups of a departure period length (kept between calls)
int gpu_groups(lpsim_assign *a, uint32_t period_steps) {
    AssignGpu *g = a->gpu;
    if (g->period_steps == period_steps) return LPSIM_OK;
    group_trips(a, period_steps, g->order, g->gstart);
    const uint64_t ng = g->gstart.size() - 1;
    std::vector<GroupRec> recs(ng);
    std::vector<uint32_t> ord(a->n);
    for (uint64_t i = 0; i < a->n; i++) ord[i] = (uint32_t)g->order[i];
    for (uint64_t q = 0; q < ng; q++) {
        const uint64_t j0 = g->order[g->gstart[q]];
        const uint64_t t0 = period_root_ms(a, a->dep[j0] / period_steps, period_steps);
        if (t0 > 0xFFFFFFFFull) return fail(LPSIM_E_INVALID_ARG, "departure period beyond the millisecond range");
        recs[q] = GroupRec{a->orig[j0], (uint32_t)t0, (uint32_t)g->gstart[q],
                           (uint32_t)(g->gstart[q + 1] - g->gstart[q])};
    }
    if (g->A.groups) g->release(const_cast<GroupRec *>(g->A.groups));
    if (g->A.order) g->release(const_cast<uint32_t *>(g->A.order));
    GroupRec *dg;
    uint32_t *dord;
    TRY(dput(g, dg, recs.data(), recs.size()));
    TRY(dput(g, dord, ord.data(), ord.size()));
    g->A.groups = dg;
    g->A.order = dord;
    g->A.n_groups = (uint32_t)ng;
    g->period_steps = period_steps;
    return LPSIM_OK;
}

}  // namespace

namespace {

// the link-time table of tt in whole milliseconds (the host searches' table) on the device
int gpu_table(lpsim_assign *a, const float *tt, uint32_t n_bins, uint32_t bin_steps) {
    AssignGpu *g = a->gpu;
    TreeArgs &A = g->A;
    const uint64_t bin_ms = table_bin_ms(a, bin_steps);
    if (bin_ms > 0xFFFFFFFFull) return fail(LPSIM_E_INVALID_ARG, "bin longer than the 32-bit millisecond range");
    static_assert(sizeof(LinkTime) == sizeof(uint2), "link-time record");
    const size_t cells = (size_t)n_bins * a->n_edges;
    // the previous call's upload of the staging table has finished (each call synchronises)
    LinkTime *tbm = g->table_buf(cells);
    if (!tbm) return fail(LPSIM_E_OOM, "host allocation of the link-time table failed");
    fill_link_times(a, tt, n_bins, bin_ms, tbm);
    if (A.cms && A.n_bins != n_bins) {
        g->release(const_cast<uint2 *>(A.cms));
        A.cms = nullptr;
    }
    if (!A.cms) {
        A.cms = static_cast<uint2 *>(g->alloc(cells * sizeof(uint2)));
        if (!A.cms) return fail(LPSIM_E_OOM, "device allocation of the link-time table failed");
    }
    CU(cudaMemcpyAsync(const_cast<uint2 *>(A.cms), tbm, cells * sizeof(uint2), cudaMemcpyHostToDevice, g->stream));
    A.n_bins = n_bins;
    A.bin_ms = (uint32_t)bin_ms;
    // the staging table is rewritten by the next call: let the copy finish first
    CU(cudaStreamSynchronize(g->stream));
    return LPSIM_OK;
}

}  // namespace

extern "C" int lpsim_assign_load_gpu(const lpsim_assign *ac, const float *tt, uint32_t n_bins, uint32_t bin_steps,
                                     uint32_t *inflow) {
    lpsim_assign *a = const_cast<lpsim_assign *>(ac);
    if (!a || !tt || !inflow || n_bins == 0 || bin_steps == 0) return fail(LPSIM_E_INVALID_ARG, "bad argument");
    if (a->n == 0) {
        std::memset(inflow, 0, (size_t)a->n_edges * n_bins * 4);
        return LPSIM_OK;
    }
    if (!a->gpu) TRY(gpu_setup(a));
    AssignGpu *g = a->gpu;
    int dev = -1;
    CU(cudaGetDevice(&dev));
    if (dev != g->device) return fail(LPSIM_E_STATE, "the device current at the first GPU call must be current");
    TRY(gpu_table(a, tt, n_bins, bin_steps));
    // the current routes, flattened (offsets on the host's threads)
    std::vector<unsigned long long> off(a->n + 1);
    off[0] = 0;
    for (uint64_t j = 0; j < a->n; j++) off[j + 1] = off[j] + a->route[j].size();
    const uint64_t total = off[a->n];
    uint32_t *edges = g->edges_buf(total);
    if (!edges) return fail(LPSIM_E_OOM, "host allocation of the route staging failed");
    lpsim::parallel_pieces(a->n, [&](uint64_t j0, uint64_t j1, uint64_t) {
        for (uint64_t j = j0; j < j1; j++) std::memcpy(edges + off[j], a->route[j].data(), a->route[j].size() * 4);
    });
    if (!g->roff) {
        g->roff = static_cast<unsigned long long *>(g->alloc((a->n + 1) * 8));
        if (!g->roff) return fail(LPSIM_E_OOM, "device allocation of the route offsets failed");
    }
    if (total > g->redge_cap) {
        if (g->redge) g->release(g->redge);
        g->redge_cap = total + total / 4;
        g->redge = static_cast<uint32_t *>(g->alloc(g->redge_cap * 4));
        if (!g->redge) return fail(LPSIM_E_OOM, "device allocation of the routes failed");
    }
    const size_t cells = (size_t)a->n_edges * n_bins;
    if (cells > g->inflow_cells) {
        if (g->inflow) g->release(g->inflow);
        g->inflow = static_cast<uint32_t *>(g->alloc(cells * 4));
        if (!g->inflow) return fail(LPSIM_E_OOM, "device allocation of the inflow table failed");
        g->inflow_cells = cells;
    }
    CU(cudaMemcpyAsync(g->roff, off.data(), (a->n + 1) * 8, cudaMemcpyHostToDevice, g->stream));
    if (total) CU(cudaMemcpyAsync(g->redge, edges, total * 4, cudaMemcpyHostToDevice, g->stream));
    CU(cudaMemsetAsync(g->inflow, 0, cells * 4, g->stream));
    load_routes<<<(unsigned)std::min<uint64_t>((a->n + 255) / 256, 65535), 256, 0, g->stream>>>(
        g->roff, g->redge, g->A.dep_ms, a->n, g->A.cms, a->n_edges, n_bins, g->A.bin_ms, g->inflow);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(inflow, g->inflow, cells * 4, cudaMemcpyDeviceToHost, g->stream));
    CU(cudaStreamSynchronize(g->stream));
    return LPSIM_OK;
}

extern "C" int lpsim_assign_shortest_paths_gpu(lpsim_assign *a, const float *tt, uint32_t n_bins, uint32_t bin_steps,
                                               uint32_t period_steps, float *t_sp) {
    if (!a || !tt || n_bins == 0 || bin_steps == 0 || period_steps == 0)
        return fail(LPSIM_E_INVALID_ARG, "bad argument");
    if (a->n == 0) return LPSIM_OK;
    if (!a->gpu) TRY(gpu_setup(a));
    AssignGpu *g = a->gpu;
    int dev = -1;
    CU(cudaGetDevice(&dev));
    if (dev != g->device) return fail(LPSIM_E_STATE, "the device current at the first GPU search must be current");
    TRY(gpu_groups(a, period_steps));
    TreeArgs &A = g->A;
    // link times in whole milliseconds, bin-major (the host searches' table)
    TRY(gpu_table(a, tt, n_bins, bin_steps));
    // path buffer: room for the current routes' length and half as much again
    if (!g->cap) {
        uint64_t total = 0;
        for (auto &r : a->route) total += r.size();
        g->cap = std::max<uint64_t>(total + total / 2, 1u << 20);
        A.edges = static_cast<uint32_t *>(g->alloc(g->cap * 4));
        if (!A.edges) return fail(LPSIM_E_OOM, "device allocation of the path buffer failed");
    }
    unsigned long long used = 0;
    uint32_t err = 0;
    for (int attempt = 0; attempt < 3; attempt++) {
        A.cap = g->cap;
        CU(cudaMemsetAsync(A.cursor, 0, 8, g->stream));
        CU(cudaMemsetAsync(A.next_group, 0, 4, g->stream));
        CU(cudaMemsetAsync(A.err, 0, 4, g->stream));
        td_trees<<<g->n_warps / kWarpsPerBlock, kWarpsPerBlock * 32, 0, g->stream>>>(A);
        CU(cudaGetLastError());
        CU(cudaMemcpyAsync(&used, A.cursor, 8, cudaMemcpyDeviceToHost, g->stream));
        CU(cudaMemcpyAsync(&err, A.err, 4, cudaMemcpyDeviceToHost, g->stream));
        CU(cudaStreamSynchronize(g->stream));
        if (!(err & kErrCapacity)) break;
        // the paths did not fit: a buffer of the length they asked for, and again
        g->release(A.edges);
        g->cap = used + used / 4 + 1024;
        A.edges = static_cast<uint32_t *>(g->alloc(g->cap * 4));
        if (!A.edges) return fail(LPSIM_E_OOM, "device allocation of the path buffer failed");
    }
    if (err & kErrBound) return fail(LPSIM_E_INVARIANT, "GPU path search exceeded its round or path-length bound");
    if (err & kErrUnreachable) return fail(LPSIM_E_INVALID_ARG, "a destination is unreachable from its origin");
    if (err & kErrCapacity) return fail(LPSIM_E_OOM, "path buffer still too small after resizing");
    std::vector<unsigned long long> off(a->n);
    std::vector<uint32_t> len(a->n);
    uint32_t *edges = g->edges_buf(used);
    if (!edges) return fail(LPSIM_E_OOM, "host allocation of the path staging failed");
    CU(cudaMemcpyAsync(off.data(), A.path_off, a->n * 8, cudaMemcpyDeviceToHost, g->stream));
    CU(cudaMemcpyAsync(len.data(), A.path_len, a->n * 4, cudaMemcpyDeviceToHost, g->stream));
    CU(cudaMemcpyAsync(a->tsp.data(), A.tsp, a->n * 4, cudaMemcpyDeviceToHost, g->stream));
    if (used) CU(cudaMemcpyAsync(edges, A.edges, used * 4, cudaMemcpyDeviceToHost, g->stream));
    CU(cudaStreamSynchronize(g->stream));
    lpsim::parallel_pieces(a->n, [&](uint64_t j0, uint64_t j1, uint64_t) {
        for (uint64_t j = j0; j < j1; j++) a->cand[j].assign(edges + off[j], edges + off[j] + len[j]);
    });
    if (t_sp) std::memcpy(t_sp, a->tsp.data(), a->n * 4);
    return LPSIM_OK;
}
