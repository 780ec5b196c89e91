/*
 * Free-flow shortest-path routing for synthetic trip tables.
 *
 * Routing is upstream of the simulation: the method takes each vehicle's
 * route as given input ("after the routing", Sec. 3.1, Network/Vehicle Data
 * Information).  This file only turns (origin node, destination node) pairs
 * into edge sequences so that the synthetic demand has realistic routes.
 *
 * Dijkstra on integer edge costs (free-flow milliseconds, computed by the
 * caller), binary heap keyed by (distance, node id).  Ties between equally
 * short paths go to the lower edge id: pred[v] is the smallest-id in-edge
 * that attains dist[v].  Integer costs make the result identical on every
 * host.  Origins are distributed over POSIX threads; each origin's tree is
 * deterministic, so the output does not depend on the thread count.  A
 * search stops once every destination of its origin's trips is settled:
 * with positive costs a settled node's distance and predecessor are final,
 * and so are those of the settled nodes on its path, so the routes are the
 * same as those of the full tree.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint64_t key; /* distance */
    uint32_t node;
} heap_item;

typedef struct {
    uint32_t n_nodes, n_edges;
    const uint32_t *src, *dst;
    const int64_t *cost;
    uint32_t *out_off, *out_edge; /* CSR of out-edges, edges ascending */
    uint64_t n_trips;
    const uint32_t *orig, *dest;
    /* trips grouped by origin */
    uint32_t *origins;       /* unique origin nodes */
    uint64_t *grp_off;       /* n_origins + 1 */
    uint64_t *grp_trip;      /* trip ids grouped */
    uint32_t n_origins;
    /* results */
    uint32_t **trip_ptr;     /* per trip: pointer into a thread buffer */
    uint32_t *trip_len;
    /* work distribution */
    uint32_t next_origin;
    pthread_mutex_t mu;
    int error;
} wl_ctx;

typedef struct {
    wl_ctx *ctx;
    uint32_t **bufs;  /* list of blocks owned by the thread */
    uint32_t n_bufs, cap_bufs;
} wl_thread;

typedef struct {
    uint64_t total;
    uint64_t n_trips;
    uint32_t **trip_ptr;
    uint32_t *trip_len;
    wl_thread *threads;
    int n_threads;
} wl_routes;

static int heap_less(const heap_item *a, const heap_item *b) {
    if (a->key != b->key) return a->key < b->key;
    return a->node < b->node;
}

static void heap_push(heap_item *h, uint64_t *n, heap_item it) {
    uint64_t i = (*n)++;
    h[i] = it;
    while (i > 0) {
        uint64_t p = (i - 1) / 2;
        if (!heap_less(&h[i], &h[p])) break;
        heap_item t = h[i]; h[i] = h[p]; h[p] = t;
        i = p;
    }
}

static heap_item heap_pop(heap_item *h, uint64_t *n) {
    heap_item top = h[0];
    h[0] = h[--(*n)];
    uint64_t i = 0;
    for (;;) {
        uint64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < *n && heap_less(&h[l], &h[m])) m = l;
        if (r < *n && heap_less(&h[r], &h[m])) m = r;
        if (m == i) break;
        heap_item t = h[i]; h[i] = h[m]; h[m] = t;
        i = m;
    }
    return top;
}

#define BLOCK_WORDS (1u << 22)

static uint32_t *thread_alloc(wl_thread *t, uint32_t words, uint32_t *used) {
    /* bump allocator over 16 MB blocks */
    if (t->n_bufs == 0 || *used + words > BLOCK_WORDS) {
        if (t->n_bufs == t->cap_bufs) {
            t->cap_bufs = t->cap_bufs ? 2 * t->cap_bufs : 16;
            t->bufs = (uint32_t **)realloc(t->bufs, t->cap_bufs * sizeof(uint32_t *));
        }
        uint32_t sz = words > BLOCK_WORDS ? words : BLOCK_WORDS;
        t->bufs[t->n_bufs++] = (uint32_t *)malloc((size_t)sz * 4);
        *used = 0;
    }
    uint32_t *p = t->bufs[t->n_bufs - 1] + *used;
    *used += words;
    return p;
}

static void *worker(void *arg) {
    wl_thread *t = (wl_thread *)arg;
    wl_ctx *c = t->ctx;
    uint32_t nn = c->n_nodes;
    uint64_t *dist = (uint64_t *)malloc((size_t)nn * 8);
    uint32_t *pred = (uint32_t *)malloc((size_t)nn * 4);
    uint8_t *done = (uint8_t *)malloc(nn);
    heap_item *heap = (heap_item *)malloc(((size_t)c->n_edges + nn + 1) * sizeof(heap_item));
    uint32_t *tmp = (uint32_t *)malloc((size_t)nn * 4 + 4);
    uint32_t *want = (uint32_t *)calloc((size_t)nn, 4);  /* origin group + 1 for its destinations */
    uint32_t used = 0;
    for (;;) {
        pthread_mutex_lock(&c->mu);
        uint32_t g = c->next_origin++;
        pthread_mutex_unlock(&c->mu);
        if (g >= c->n_origins) break;
        uint32_t s = c->origins[g];
        uint32_t n_want = 0;
        for (uint64_t j = c->grp_off[g]; j < c->grp_off[g + 1]; j++) {
            uint32_t d = c->dest[c->grp_trip[j]];
            if (want[d] != g + 1) { want[d] = g + 1; n_want++; }
        }
        for (uint32_t i = 0; i < nn; i++) { dist[i] = UINT64_MAX; pred[i] = UINT32_MAX; done[i] = 0; }
        uint64_t hn = 0;
        dist[s] = 0;
        heap_push(heap, &hn, (heap_item){0, s});
        while (hn) {
            heap_item it = heap_pop(heap, &hn);
            uint32_t u = it.node;
            if (done[u] || it.key != dist[u]) continue;
            done[u] = 1;
            if (want[u] == g + 1 && --n_want == 0) break;
            for (uint32_t j = c->out_off[u]; j < c->out_off[u + 1]; j++) {
                uint32_t e = c->out_edge[j];
                uint32_t v = c->dst[e];
                if (done[v]) continue;
                uint64_t nd = dist[u] + (uint64_t)c->cost[e];
                if (nd < dist[v]) {
                    dist[v] = nd; pred[v] = e;
                    heap_push(heap, &hn, (heap_item){nd, v});
                } else if (nd == dist[v] && e < pred[v]) {
                    pred[v] = e;
                }
            }
        }
        for (uint64_t j = c->grp_off[g]; j < c->grp_off[g + 1]; j++) {
            uint64_t trip = c->grp_trip[j];
            uint32_t d = c->dest[trip];
            uint32_t len = 0, v = d;
            if (d == s || dist[d] == UINT64_MAX) { c->error = 1; c->trip_len[trip] = 0; continue; }
            while (v != s) { uint32_t e = pred[v]; tmp[len++] = e; v = c->src[e]; }
            uint32_t *p = thread_alloc(t, len, &used);
            for (uint32_t q = 0; q < len; q++) p[q] = tmp[len - 1 - q];
            c->trip_ptr[trip] = p;
            c->trip_len[trip] = len;
        }
    }
    free(dist); free(pred); free(done); free(heap); free(tmp); free(want);
    return NULL;
}

/* Route every trip; returns a handle (NULL on allocation failure).  *status is
 * 0 on success, 1 if some destination was unreachable or equal to its origin
 * (those trips get empty routes), 2 on bad arguments. */
void *wl_route(uint32_t n_nodes, uint32_t n_edges, const uint32_t *src, const uint32_t *dst,
               const int64_t *cost, uint64_t n_trips, const uint32_t *orig, const uint32_t *dest,
               int n_threads, int *status) {
    *status = 0;
    for (uint32_t e = 0; e < n_edges; e++)
        if (src[e] >= n_nodes || dst[e] >= n_nodes || cost[e] <= 0) { *status = 2; return NULL; }
    for (uint64_t i = 0; i < n_trips; i++)
        if (orig[i] >= n_nodes || dest[i] >= n_nodes) { *status = 2; return NULL; }
    wl_ctx c;
    memset(&c, 0, sizeof c);
    c.n_nodes = n_nodes; c.n_edges = n_edges; c.src = src; c.dst = dst; c.cost = cost;
    c.n_trips = n_trips; c.orig = orig; c.dest = dest;
    c.out_off = (uint32_t *)calloc((size_t)n_nodes + 1, 4);
    c.out_edge = (uint32_t *)malloc((size_t)n_edges * 4 + 4);
    for (uint32_t e = 0; e < n_edges; e++) c.out_off[src[e] + 1]++;
    for (uint32_t i = 0; i < n_nodes; i++) c.out_off[i + 1] += c.out_off[i];
    uint32_t *fill = (uint32_t *)malloc((size_t)n_nodes * 4 + 4);
    memcpy(fill, c.out_off, (size_t)n_nodes * 4);
    for (uint32_t e = 0; e < n_edges; e++) c.out_edge[fill[src[e]]++] = e; /* ascending ids */
    /* group trips by origin (counting sort, stable) */
    uint64_t *cnt = (uint64_t *)calloc((size_t)n_nodes + 1, 8);
    for (uint64_t i = 0; i < n_trips; i++) cnt[orig[i] + 1]++;
    uint32_t n_org = 0;
    for (uint32_t i = 0; i < n_nodes; i++) if (cnt[i + 1]) n_org++;
    c.origins = (uint32_t *)malloc((size_t)n_org * 4 + 4);
    c.grp_off = (uint64_t *)malloc(((size_t)n_org + 1) * 8);
    c.grp_trip = (uint64_t *)malloc((size_t)n_trips * 8 + 8);
    uint64_t *pos = (uint64_t *)malloc((size_t)n_nodes * 8 + 8);
    uint32_t g = 0; uint64_t acc = 0;
    for (uint32_t i = 0; i < n_nodes; i++) {
        pos[i] = acc;
        if (cnt[i + 1]) { c.origins[g] = i; c.grp_off[g] = acc; g++; acc += cnt[i + 1]; }
    }
    c.grp_off[n_org] = acc;
    for (uint64_t i = 0; i < n_trips; i++) c.grp_trip[pos[orig[i]]++] = i;
    c.n_origins = n_org;
    c.trip_ptr = (uint32_t **)calloc((size_t)n_trips + 1, sizeof(uint32_t *));
    c.trip_len = (uint32_t *)calloc((size_t)n_trips + 1, 4);
    pthread_mutex_init(&c.mu, NULL);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    wl_routes *r = (wl_routes *)calloc(1, sizeof(wl_routes));
    r->threads = (wl_thread *)calloc((size_t)n_threads, sizeof(wl_thread));
    r->n_threads = n_threads;
    pthread_t tid[256];
    for (int i = 0; i < n_threads; i++) {
        r->threads[i].ctx = &c;
        pthread_create(&tid[i], NULL, worker, &r->threads[i]);
    }
    for (int i = 0; i < n_threads; i++) pthread_join(tid[i], NULL);
    pthread_mutex_destroy(&c.mu);
    r->n_trips = n_trips;
    r->trip_ptr = c.trip_ptr;
    r->trip_len = c.trip_len;
    r->total = 0;
    for (uint64_t i = 0; i < n_trips; i++) r->total += c.trip_len[i];
    if (c.error) *status = 1;
    free(c.out_off); free(c.out_edge); free(fill); free(cnt); free(c.origins);
    free(c.grp_off); free(c.grp_trip); free(pos);
    return r;
}

uint64_t wl_route_total(void *h) { return ((wl_routes *)h)->total; }

void wl_route_copy(void *h, uint64_t *off, uint32_t *edges) {
    wl_routes *r = (wl_routes *)h;
    uint64_t acc = 0;
    for (uint64_t i = 0; i < r->n_trips; i++) {
        off[i] = acc;
        if (r->trip_len[i]) memcpy(edges + acc, r->trip_ptr[i], (size_t)r->trip_len[i] * 4);
        acc += r->trip_len[i];
    }
    off[r->n_trips] = acc;
}

void wl_route_free(void *h) {
    wl_routes *r = (wl_routes *)h;
    for (int i = 0; i < r->n_threads; i++) {
        for (uint32_t b = 0; b < r->threads[i].n_bufs; b++) free(r->threads[i].bufs[b]);
        free(r->threads[i].bufs);
    }
    free(r->threads); free(r->trip_ptr); free(r->trip_len); free(r);
}
