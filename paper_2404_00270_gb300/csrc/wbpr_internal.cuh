// Internal types shared by the translation units of the WBPR library.
//
// Device data layout (one handle = one graph instance):
//   BCSR (§3.2, Fig. 2(d)): off[n+1] (int64) rows of merged, id-sorted
//     neighbour lists; per slot a: col[a] (int32 neighbour), cf[a] (int32
//     residual capacity of the arc row(a) -> col[a]), cf0[a] (its initial
//     value), rev[a] (uint32 slot of the paired entry in col[a]'s row),
//     cfb[a] (= cf[rev[a]], the reverse residual mirrored in place).
//   RCSR (§3.2, Fig. 2(c)): off[n+1] out rows, per out slot j: col[j] (head),
//     cf[j] (forward residual), bf[j] (backward residual = flow on arc j),
//     cf0[j] (capacity); in_off[n+1] in rows, per in slot k: in_col[k]
//     (tail), flow_idx[k] (the out slot j of the same arc).
//   Per vertex: e[n] (int64 excess), h[n] (int32 height), dead[n] (uint8:
//     excess already written off), count[n+1] (int32 vertices per height,
//     gap heuristic), six int32[n] queues (2 generations x 3 tile classes).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "wbpr.h"

namespace wbpr {

constexpr int kBlock = 256;         // threads per block of the persistent solver
constexpr int kWarps = kBlock / 32;
constexpr int kClasses = 3;         // tile classes: small tile, warp, block
constexpr int kQueueCap = 1024;     // per-class shared-memory staging of queue appends
constexpr int kUnvisited = 0x7fffffff;
constexpr long long kRenumberAutoVertices = 1LL << 22;  // renumber = -1: on from this many vertices
#ifndef WBPR_WCHUNK
#define WBPR_WCHUNK 256
#endif
constexpr int kWChunk = WBPR_WCHUNK;  // hub rows (push-relabel passes, BFS levels, the cut): chunks of
                                      // this many entries, one per warp (kWChunk / 32 per lane), taken
                                      // dynamically
// Staging of push-relabel hub chunks in shared memory: per warp two buffers
// of kWChunk entries (neighbour ids and residual capacities).
constexpr int kStageInts = 2 * 2 * WBPR_WCHUNK;            // per warp
constexpr int kStageBytes = (kBlock / 32) * kStageInts * 4;  // per block (dynamic shared memory)

enum Layout : int { kRCSR = 0, kBCSR = 1 };

// Per-block statistics slots (reduced on the host after a launch).
enum Stat : int {
    kStatPushes = 0,
    kStatRelabels,
    kStatArcs,
    kStatGrArcs,
    kStatActive,
    kStatGaps,
    kStatAvqFull,    // AVQ compactions that scanned every vertex
    kStatAvqInc,     // AVQ compactions from the candidate bitmap
    kStatAvqCand,    // candidates those examined
    kStatCount
};

// Device control block, cleared before every solver launch.
struct __align__(128) Ctl {
    unsigned long long bar;  // grid barrier: total arrivals
    unsigned long long pad0[15];
    int err;                 // wbpr_status of a device-side failure (0 = none)
    int err_where;           // which wait gave up
    int gap_level[3];        // lowest emptied height level, by queue generation % 3
    int pad1;
    long long excess_total;  // Excess_total of Alg. 1
    long long preflow_total; // excess created by the preflow
    long long written_off;
    long long iterations;
    long long phase1_iterations;
    long long global_relabels;
    long long cut_value;
    unsigned q_count[3][kClasses];  // queue sizes by generation % 3 and class (0, 1)
    unsigned q_grab[3];             // dynamic work counter of the hub chunks
    unsigned q_grab_w[3];           // dynamic work counter of the warp-class rows
    unsigned long long hub_pack[3]; // hub class: (count << 40) | total chunks
    int done;
    unsigned trace_len;
    int gr_due_gen;      // time-balanced trigger: generation whose iteration made a
                         // global relabel due (-1 = none)
    int pad2;
    long long dead_count;    // vertices marked unreachable (dead[]) in the current phase
    long long dead_edges;    // their residual-list entries
    long long fedges[3];     // residual-list entries of the BFS frontier, by generation % 3
    unsigned local_active[3];  // block-local passes: active vertices processed, by generation % 3
    int local_defer[3];        // block-local passes: candidates left marked for a full pass
};

struct GraphDev {
    int n, s, t;
    int layout_tag;             // kRCSR or kBCSR (batch kernels check it)
    long long slots;
    const long long *off;
    const int *col;
    int *cf;
    const int *cf0;
    const unsigned *rev;        // BCSR, may be null when use_rev = 0
    int *cfb;                   // BCSR with rev: cfb[a] mirrors cf[rev[a]] (residual of the
                                // reverse arc, kept in place so BFS reads it coalesced); or null
    int *bf;                    // RCSR
    const long long *in_off;    // RCSR
    const int *in_col;          // RCSR
    const unsigned *flow_idx;   // RCSR
    const int *order;           // renumbered handle: solver id -> input id; or null
    const int *perm;            // renumbered handle: input id -> solver id (cut side output); or null
};

// Upper bound on the hub chunks of one queue generation: a hub of degree d
// has at most d / kWChunk + 2 chunks (the first one may start up to 3 slots
// before the row, so that lanes read aligned 16-byte vectors), and the
// degrees sum to the residual-list entries.
constexpr long long hub_chunk_entries(long long n, long long slots, int layout_tag)
{
    return 2 * n + (layout_tag == kRCSR ? 2 * slots : slots) / kWChunk + 1;
}

struct StateDev {
    long long *e;
    int *h;
    unsigned char *dead;
    int *count;
    int *q[2][kClasses];
    // per hub queue position (two generation sets): first chunk id, excess at
    // compaction, excess not yet taken by a chunk, min key / min residual height,
    // chunks finished
    unsigned *hub_start[2];
    unsigned *hub_chunk[2];     // chunk id -> hub queue position; hub_chunk_entries(n, slots, L) each
    long long *hub_e0[2];
    long long *hub_rem[2];
    unsigned long long *hub_aux[2];
    unsigned *hub_done[2];
    // one bit per vertex: pushed into, or left with excess by its owner,
    // during the last push-relabel pass (candidates of the next AVQ); null =
    // every AVQ compaction scans all vertices
    unsigned *touch;
    Ctl *ctl;
    long long *bstats;          // [gridDim.x][kStatCount]
};

// Solver launch modes (bit mask).
enum Mode : int {
    kModePreflow = 1,       // reset residual graph and state, then preflow
    kModePhase1 = 2,        // global relabel + iterations until e(s)+e(t) >= Excess_total
    kModeGrOnce = 4,        // one global relabel (phase 1 semantics)
    kModeIters = 8,         // `iters_arg` iterations, no global relabel
    kModePhase2 = 16,       // return stranded excess to s
    kModeCut = 32           // forward BFS from s: source side and cut capacity
};

struct Params {
    GraphDev g;
    StateDev st;
    int mode;
    long long iters_arg;
    int cycle;
    float gr_ratio;              // > 0: global relabel once iterations took gr_ratio x its time
    int gap;
    int use_rev;
    int multi_push;
    int small_max;
    int warp_max;
    int bottom_up;               // > 0: bottom-up BFS levels when frontier * bottom_up >=
                                 //      unvisited vertices
    int bottom_up_min;           //      and frontier >= bottom_up_min
    int bottom_up_edges;         // 1: compare the frontier's entries, not its vertices
    long long max_iterations;
    unsigned long long timeout_ns;
    unsigned char *source_side;  // kModeCut output (device, n bytes) or null
    unsigned long long *trace;   // optional: 4 words per grid barrier (where, gen, ns, queue total)
    int trace_cap;               // records
    int mirror_gather;           // reset cfb[a] = cf0[rev[a]] by gather (cf and cfb may hold another
                                 // graph's state) instead of from the pair invariant
    int thread_centric;          // 1: thread-centric iterations (one thread per vertex, no AVQ)
    unsigned long long *warp_ns; // optional: per warp of the grid, device ns spent in push-relabel passes
    int barrier_extra;           // tests: arrivals a grid barrier waits for beyond the grid
    int local_passes;            // 1: small AVQs are compacted and processed block by block (with touch)
};

// Persistent server (solver.cu).  The rings, results, published counts and
// stop flag live in host-mapped pinned memory (device pointers here).
struct ServerOut {
    long long value;
    long long iterations;
    unsigned long long t_start, t_end;  // globaltimer ns
    int err;
    int done;                           // written last (release, system scope)
};
struct ServerDesc {
    const Params *ring[2];
    ServerOut *out[2];
    const unsigned *avail[2];
    const int *stop;
    unsigned *next[2];
    unsigned long long *team_bar;
    unsigned *team_item;
    unsigned *mirror;        // device copies (u64 each): avail[0] at +0, avail[1] at +2, stop at +4
    int *poll_token;         // 1 while one leader refreshes the mirror from host memory
    int *team_exit;          // why each team left: 1 ring end, 2 stop, 3 idle, 4-6 team barrier limit
    unsigned capacity[2];
    int team_big;
    int n_big_teams;
    unsigned long long idle_ns;
    unsigned long long timeout_ns;
};
cudaError_t server_max_blocks_per_sm(int layout, int *blocks, bool build_room);
cudaError_t server_launch(int layout, int grid, const ServerDesc &d, cudaStream_t stream, bool build_room);

// Launch helpers implemented in solver.cu.
cudaError_t solver_max_blocks_per_sm(int layout, int small_tile, int *blocks, size_t dyn_smem = 0);
cudaError_t solver_launch(int layout, int small_tile, int grid, const Params &p,
                          cudaStream_t stream, size_t dyn_smem = 0);

// Edge-flow kernels (solver.cu).
cudaError_t launch_edge_flow(int layout, long long m, const unsigned *arc2slot,
                             const int *cf0, const int *cf, const int *bf, const int *prefix,
                             const int *cap_in, int *edge_flow, cudaStream_t stream);

}  // namespace wbpr
