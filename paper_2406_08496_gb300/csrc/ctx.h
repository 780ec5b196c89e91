// Internal definition of the library context (include/lpsim.h keeps it
// opaque).  Shared by the translation units of liblpsim.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lpsim.h"
#include "lpsim_dev.cuh"

// record `msg` as the calling thread's lpsim_last_error() and return `code`
int lpsim_fail(int code, const std::string &msg);

struct lpsim_ctx {
    int device = 0;
    int n_sm = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    lpsim_params p{};
    uint32_t n_nodes = 0, n_edges = 0;
    // allocation
    void *(*alloc)(size_t, void *) = nullptr;
    void (*release)(void *, void *) = nullptr;
    void *alloc_user = nullptr;
    std::vector<void *> blocks;
    // host mirror of the layout (queries)
    std::vector<uint32_t> moff;
    std::vector<uint16_t> len;
    std::vector<uint8_t> lanes;
    std::vector<uint32_t> src, dst;
    uint64_t map_bytes = 0, canon_cells = 0, lane_slots = 0;
    // device state
    lpsim::Dev d{};
    lpsim::Slots sets[2]{};
    int cur = 0;
    lpsim::SortWork w{};
    bool loaded = false;
    uint64_t n_trips = 0;
    uint32_t k = 0;
    uint32_t R = 64, C = 384;
    int grid = 0, block = 256;
    bool sort = true;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    unsigned long long *h_ctr = nullptr;  // pinned: ctr[0..7], err, n_slots, ...
    uint32_t *d_tmp = nullptr;
    lpsim::QRec *org_hd0 = nullptr;  // first trip of each origin queue (reset)
    uint64_t launches = 0;
    uint64_t stall_steps = 0;
    unsigned long long last_progress = 0;
    std::vector<uint32_t> dep_sorted;  // departure step by vehicle id (nondecreasing)
    uint32_t *small_list = nullptr;    // light-load chunks: origin edges that can act, and their count
    uint32_t *small_n = nullptr;
    uint64_t light_chunks = 0;
    uint64_t skipped = 0;              // idle steps jumped over (nothing on the network)
    // device buffers whose contents change while stepping (snapshot / restore)
    std::vector<std::pair<void *, size_t>> mut;
    uint8_t *snap = nullptr;
    size_t snap_bytes = 0;
    bool has_snap = false;
    struct {
        uint32_t k;
        int cur;
        uint64_t stall_steps;
        unsigned long long last_progress;
    } snap_host{};
    // vehicle types (lpsim_set_vehicle_types), uploaded with the trips
    std::vector<lpsim_vehicle_type> types;
    // batched scenarios: prefix offsets of nodes, edges, canonical lane-map cells and trips
    std::vector<uint64_t> scen_node_off, scen_edge_off, scen_cell_off, scen_trip_off;
    // per-kernel timing: device spans stamped by the kernels themselves
    // (d.tspan, d.tacc; see lpsim_dev.cuh), room for tspan_steps steps
    bool timing = false;
    unsigned long long *tspan_buf = nullptr;  // d.tspan while timing is on
    uint32_t tspan_steps = 0;

    void *dalloc(size_t bytes) {
        if (bytes == 0) bytes = 16;
        bytes = (bytes + 255) & ~size_t(255);
        void *ptr = nullptr;
        if (alloc) {
            ptr = alloc(bytes, alloc_user);
        } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
            ptr = nullptr;
        }
        if (ptr) blocks.push_back(ptr);
        return ptr;
    }
    ~lpsim_ctx() {
        for (int i = 0; i < 2; i++)
            if (graph[i]) cudaGraphExecDestroy(graph[i]);
        if (stream) cudaStreamSynchronize(stream);
        for (void *b : blocks) {
            if (release) release(b, alloc_user);
            else cudaFree(b);
        }
        if (h_ctr) cudaFreeHost(h_ctr);
        if (own_stream) cudaStreamDestroy(stream);
    }
};

