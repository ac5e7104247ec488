// Host-side handle of one graph instance (the opaque wbpr_graph of wbpr.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "wbpr.h"
#include "wbpr_internal.cuh"

namespace wbpr {

// Device allocation through the allocator hook (api.cu).  Returns null on
// failure.  `owner` (optional) records the free function in force at
// allocation time, so a block is always returned to the allocator that made
// it even if the hook changes in between.
struct DevFree {
    wbpr_free_fn fn;
    void *ctx;
};
void *dev_alloc(size_t bytes, cudaStream_t stream, DevFree *owner = nullptr);
void dev_free(void *p, size_t bytes, cudaStream_t stream, const DevFree *owner = nullptr);

// Records a failure for wbpr_last_error()/wbpr_last_error_message().
wbpr_status set_error(wbpr_status st, const std::string &msg);

}  // namespace wbpr

struct wbpr_graph {
    int64_t n = 0, m = 0;
    int32_t s = 0, t = 0;     // as given (input ids)
    int32_t s_int = 0, t_int = 0;  // the solver's ids (differ when renumbered)
    bool renumbered = false;  // vertices renumbered by the builder (order != null)
    bool lean = false;        // lean build: sort blocks that fit beside a resident server
    int32_t layout = 0;
    int64_t slots = 0;        // BCSR merged entries / RCSR arcs without loops
    int64_t mprime = 0;       // input arcs that are not self-loops
    int64_t max_degree = 0;
    int device = 0;
    int num_sms = 0;
    int grid_blocks = 0;      // persistent grid of the last solve
    wbpr_options opts;
    wbpr_stats stats;
    bool solved_flow = false; // phase 2 done on the current state
    bool solved_value = false;

    // graph (device)
    int *order = nullptr;     // renumbered: solver id -> input id
    int *perm = nullptr;      // renumbered: input id -> solver id
    long long *off = nullptr;
    int *col = nullptr;
    int *cf = nullptr;
    int *cf0 = nullptr;
    unsigned *rev = nullptr;
    int *cfb = nullptr;       // BCSR: mirrored reverse residual
    int *bf = nullptr;
    long long *in_off = nullptr;
    int *in_col = nullptr;
    unsigned *flow_idx = nullptr;
    unsigned *arc2slot = nullptr;
    int *prefix = nullptr;    // BCSR: capacity of earlier duplicates of each input arc
    int *cap_in = nullptr;    // BCSR: input capacities (edge-flow split)
    // solver state (device)
    long long *e = nullptr;
    int *h = nullptr;
    unsigned char *dead = nullptr;
    int *count = nullptr;
    int *q[2][wbpr::kClasses] = {{nullptr}};
    unsigned *hub_start[2] = {nullptr, nullptr};
    unsigned *hub_chunk[2] = {nullptr, nullptr};  // chunk id -> hub queue position
    long long *hub_e0[2] = {nullptr, nullptr};
    long long *hub_rem[2] = {nullptr, nullptr};
    unsigned long long *hub_aux[2] = {nullptr, nullptr};
    unsigned *hub_done[2] = {nullptr, nullptr};
    unsigned *touch = nullptr;
    wbpr::Ctl *ctl = nullptr;
    long long *bstats = nullptr;
    unsigned long long *trace = nullptr;  // optional barrier trace (wbpr_options.trace)
    unsigned long long *warp_ns = nullptr;  // optional per-warp busy time (wbpr_options.warp_time)
    int trace_cap = 0;
    int bstats_blocks = 0;
    int *edge_tmp = nullptr;           // device staging of edge flows for host outputs
    unsigned char *side_tmp = nullptr; // device staging of the cut side for host outputs
    // host
    long long *pinned = nullptr;       // host staging of small results (64 words)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;

    struct Block {
        void *p;
        size_t bytes;
        wbpr::DevFree owner;
    };
    std::vector<Block> blocks;  // every device allocation owned by the handle
    int64_t device_bytes = 0;

    void *alloc(size_t bytes, cudaStream_t st)
    {
        if (bytes == 0) bytes = 16;
        wbpr::DevFree owner;
        void *p = wbpr::dev_alloc(bytes, st, &owner);
        if (p) {
            blocks.push_back({p, bytes, owner});
            device_bytes += (int64_t)bytes;
        }
        return p;
    }
};

namespace wbpr {
// Graph builders (builder.cu).  The inputs are device pointers.
wbpr_status build_graph(wbpr_graph *g, const int *src, const int *dst, const int *cap,
                        cudaStream_t stream);
// Solver parameters of a handle for the given launch modes (api.cu).
Params make_params(wbpr_graph *g, int mode);
}  // namespace wbpr
