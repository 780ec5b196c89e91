// Compaction of the vehicle slots and on-device LSD radix sort by lane-map
// cell.
//
// Vehicles live in slots; a slot whose vehicle arrived is a hole until the
// next compaction.  Every `sort_period` steps the live slots are packed
// (stable prefix sum over tiles) and, when sorting, ordered by the global
// lane-map cell they occupy: vehicles of one lane row become neighbours in
// slot order, so a warp's leader scans read neighbouring bytes and its state
// loads are contiguous.  The paper sorts trips by departure time to cut
// divergence (Sec. 4, Table 6); cells are unique per vehicle, so this order
// is a total order and the results do not depend on it anyway.
//
// Kernels: tile_count -> tile_scan -> (scatter | key scatter -> radix passes
// -> gather).  Tiles of 2048 slots, 256 threads x 8 items.
#include "lpsim_dev.cuh"

namespace lpsim {

namespace {

constexpr int kBlock = 256;
constexpr int kItems = 8;
constexpr uint32_t kTile = kBlock * kItems;

__device__ __forceinline__ uint32_t n_src(const SortWork &w) { return w.tile_off[w.max_tiles + 1]; }

// live slots per tile; arrived slots get their last cell erased here
__global__ void __launch_bounds__(kBlock) tile_count(Dev d, SortWork w, uint32_t koff) {
    span_start(d, 3 * koff + 2);
    const uint32_t k = *d.kbase + koff;
    const uint32_t n = *d.n_slots;
    const uint32_t ntiles = (n + kTile - 1) / kTile;
    uint8_t *Mk = d.map[k % 3];
    __shared__ uint32_t red[kBlock / 32];
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        uint32_t cnt = 0;
#pragma unroll
        for (int j = 0; j < kItems; j++) {
            uint32_t s = t * kTile + j * kBlock + threadIdx.x;
            if (s < n) {
                uint8_t f = d.s.flag[s];
                if (f == kLive) cnt++;
                else if (f == kArrivedPending) {
                    uint32_t pc = d.s.pcell[s];
                    if (pc != kNone) Mk[pc] = kEmpty;
                }
            }
        }
        cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tot = 0;
            for (int q = 0; q < kBlock / 32; q++) tot += red[q];
            w.tile_cnt[t] = tot;
        }
        __syncthreads();
    }
}

// exclusive scan of the tile counts (one block); publishes the new slot count
__global__ void __launch_bounds__(1024) tile_scan(Dev d, SortWork w) {
    const uint32_t n = *d.n_slots;
    const uint32_t ntiles = (n + kTile - 1) / kTile;
    __shared__ uint32_t warp_sum[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < ntiles; base += 1024) {
        uint32_t t = base + threadIdx.x;
        uint32_t v = t < ntiles ? w.tile_cnt[t] : 0u;
        uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        uint32_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        if (lane == 31) warp_sum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            uint32_t s = warp_sum[lane];
            uint32_t si = s;
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xFFFFFFFFu, si, o);
                if (lane >= (uint32_t)o) si += y;
            }
            warp_sum[lane] = si - s;  // exclusive over warps
        }
        __syncthreads();
        uint32_t excl = carry + warp_sum[wid] + incl - v;
        if (t < ntiles) w.tile_off[t] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        w.tile_off[w.max_tiles] = carry;      // live slots
        w.tile_off[w.max_tiles + 1] = n;      // slots before compaction
        *d.n_slots = carry;
    }
}

// in-tile exclusive rank of the live slots, in slot order
__device__ __forceinline__ void tile_ranks(const uint8_t *flag, uint32_t t, uint32_t n, bool live[kItems],
                                           uint32_t rank[kItems]) {
    __shared__ uint32_t wsum[kBlock / 32];
    // thread owns items t*kTile + threadIdx.x*kItems + j (contiguous)
    uint32_t cnt = 0;
#pragma unroll
    for (int j = 0; j < kItems; j++) {
        uint32_t s = t * kTile + threadIdx.x * kItems + j;
        live[j] = s < n && flag[s] == kLive;
        rank[j] = cnt;
        cnt += live[j];
    }
    uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= (uint32_t)o) incl += y;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    uint32_t woff = 0;
    for (uint32_t q = 0; q < wid; q++) woff += wsum[q];
    uint32_t excl = woff + incl - cnt;
#pragma unroll
    for (int j = 0; j < kItems; j++) rank[j] += excl;
    __syncthreads();
}

__device__ __forceinline__ void copy_slot(const Slots &a, uint32_t s, const Slots &b, uint32_t o, int par) {
    reinterpret_cast<uint4 *>(b.es + o)[0] = reinterpret_cast<const uint4 *>(a.es + s)[0];
    reinterpret_cast<uint4 *>(b.es + o)[1] = reinterpret_cast<const uint4 *>(a.es + s)[1];
    b.id[o] = a.id[s];
    b.rlast[o] = a.rlast[s];
    b.tent[o] = a.tent[s];
    b.pcell[o] = a.pcell[s];
    b.imark[o] = a.imark[s];
    b.cprev[o] = a.cprev[s];
    b.lane[o] = a.lane[s];
    b.tlc[o] = a.tlc[s];
    b.flag[o] = kLive;
    b.x[par][o] = a.x[par][s];
    b.v[par][o] = a.v[par][s];
}

// plain compaction: live slots of the current set into `dst`, same order
__global__ void __launch_bounds__(kBlock) scatter_slots(Dev d, Slots dst, SortWork w, uint32_t koff) {
    const uint32_t k = *d.kbase + koff;
    const uint32_t n = n_src(w);
    const uint32_t ntiles = (n + kTile - 1) / kTile;
    const int par = (k + 1) & 1;
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        bool live[kItems];
        uint32_t rank[kItems];
        tile_ranks(d.s.flag, t, n, live, rank);
        const uint32_t off = w.tile_off[t];
#pragma unroll
        for (int j = 0; j < kItems; j++)
            if (live[j]) copy_slot(d.s, t * kTile + threadIdx.x * kItems + j, dst, off + rank[j], par);
    }
    span_end(d, 3 * koff + 2);
}

// sort keys: the cell each live vehicle occupies in the map of step k+1
__global__ void __launch_bounds__(kBlock) scatter_keys(Dev d, SortWork w, uint32_t koff) {
    const uint32_t k = *d.kbase + koff;
    const uint32_t n = n_src(w);
    const uint32_t ntiles = (n + kTile - 1) / kTile;
    const float *x = d.s.x[(k + 1) & 1];
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        bool live[kItems];
        uint32_t rank[kItems];
        tile_ranks(d.s.flag, t, n, live, rank);
        const uint32_t off = w.tile_off[t];
#pragma unroll
        for (int j = 0; j < kItems; j++) {
            if (!live[j]) continue;
            uint32_t s = t * kTile + threadIdx.x * kItems + j;
            w.key[0][off + rank[j]] = d.s.es[s].base + (uint32_t)x[s];
            w.perm[0][off + rank[j]] = s;
        }
    }
}

// ------------------------------------------------------------ radix passes

__global__ void __launch_bounds__(kBlock) radix_hist(Dev d, SortWork w, int in, uint32_t shift) {
    const uint32_t n = *d.n_slots;
    const uint32_t ntiles = (n + kTile - 1) / kTile;
    __shared__ uint32_t h[256];
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        h[threadIdx.x] = 0;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kItems; j++) {
            uint32_t i = t * kTile + j * kBlock + threadIdx.x;
            if (i < n) atomicAdd(&h[(w.key[in][i] >> shift) & 255u], 1u);
        }
        __syncthreads();
        w.hist[threadIdx.x * ntiles + t] = h[threadIdx.x];
        __syncthreads();
    }
}

// exclusive scan over hist[digit][tile] in digit-major order (one block)
__global__ void __launch_bounds__(1024) radix_scan(Dev d, SortWork w) {
    const uint32_t n = *d.n_slots;
    const uint32_t ntiles = (n + kTile - 1) / kTile;
    const uint32_t total = 256u * ntiles;
    __shared__ uint32_t warp_sum[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < total; base += 1024) {
        uint32_t t = base + threadIdx.x;
        uint32_t v = t < total ? w.hist[t] : 0u;
        uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        uint32_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        if (lane == 31) warp_sum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            uint32_t s = warp_sum[lane];
            uint32_t si = s;
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xFFFFFFFFu, si, o);
                if (lane >= (uint32_t)o) si += y;
            }
            warp_sum[lane] = si - s;
        }
        __syncthreads();
        uint32_t excl = carry + warp_sum[wid] + incl - v;
        if (t < total) w.hist[t] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
}

// stable scatter: rank of each key among equal digits of its tile, in order
__global__ void __launch_bounds__(kBlock) radix_scatter(Dev d, SortWork w, int in, uint32_t shift) {
    const uint32_t n = *d.n_slots;
    const uint32_t ntiles = (n + kTile - 1) / kTile;
    __shared__ uint32_t run[256];            // keys of each digit already placed in this tile
    __shared__ uint32_t wcnt[kBlock / 32][256];
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int out = in ^ 1;
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        run[threadIdx.x] = 0;
        for (int j = 0; j < kItems; j++) {
            // round j: keys t*kTile + j*kBlock + threadIdx.x, in thread order
            for (int q = 0; q < kBlock / 32; q++) wcnt[q][threadIdx.x] = 0;
            __syncthreads();
            uint32_t i = t * kTile + j * kBlock + threadIdx.x;
            bool valid = i < n;
            uint32_t key = valid ? w.key[in][i] : 0u;
            uint32_t val = valid ? w.perm[in][i] : 0u;
            uint32_t dig = valid ? (key >> shift) & 255u : 256u + lane;  // invalid lanes match nobody
            uint32_t peers = __match_any_sync(0xFFFFFFFFu, dig);
            uint32_t rank_w = __popc(peers & ((1u << lane) - 1u));
            if (valid && rank_w == 0) wcnt[wid][dig] = __popc(peers);
            __syncthreads();
            // per digit: exclusive prefix over warps, then advance the running count
            {
                uint32_t dg = threadIdx.x, acc = run[dg];
                for (int q = 0; q < kBlock / 32; q++) {
                    uint32_t c = wcnt[q][dg];
                    wcnt[q][dg] = acc;
                    acc += c;
                }
                run[dg] = acc;
            }
            __syncthreads();
            if (valid) {
                uint32_t pos = w.hist[dig * ntiles + t] + wcnt[wid][dig] + rank_w;
                w.key[out][pos] = key;
                w.perm[out][pos] = val;
            }
            __syncthreads();
        }
    }
}

// final gather of the slot state in sorted order
__global__ void __launch_bounds__(kBlock) gather_slots(Dev d, Slots dst, SortWork w, int in, uint32_t koff) {
    const uint32_t k = *d.kbase + koff;
    const uint32_t n = *d.n_slots;
    const int par = (k + 1) & 1;
    for (uint32_t i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock)
        copy_slot(d.s, w.perm[in][i], dst, i, par);
    span_end(d, 3 * koff + 2);
}

}  // namespace

int launch_compact(const Dev &d, const Slots &dst, const SortWork &w, uint32_t koff, bool sort, int grid,
                   cudaStream_t st) {
    int launches = 0;
    tile_count<<<grid, kBlock, 0, st>>>(d, w, koff);
    tile_scan<<<1, 1024, 0, st>>>(d, w);
    launches += 2;
    if (!sort) {
        scatter_slots<<<grid, kBlock, 0, st>>>(d, dst, w, koff);
        return launches + 1;
    }
    scatter_keys<<<grid, kBlock, 0, st>>>(d, w, koff);
    launches++;
    int in = 0;
    for (uint32_t shift = 0; shift < w.key_bits; shift += 8) {
        radix_hist<<<grid, kBlock, 0, st>>>(d, w, in, shift);
        radix_scan<<<1, 1024, 0, st>>>(d, w);
        radix_scatter<<<grid, kBlock, 0, st>>>(d, w, in, shift);
        in ^= 1;
        launches += 3;
    }
    gather_slots<<<grid, kBlock, 0, st>>>(d, dst, w, in, koff);
    return launches + 1;
}

uint32_t compact_tile() { return kTile; }

}  // namespace lpsim
