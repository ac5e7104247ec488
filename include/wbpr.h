/*
 * wbpr.h -- C ABI of the GB300 workload-balanced push-relabel (WBPR) library.
 *
 * The library computes a maximum s-t flow and a minimum s-t cut of a directed
 * graph with integer capacities (the problem of paper §2.1) on one CUDA GPU.
 * The method is the lock-free push-relabel algorithm of Alg. 1 run in the
 * vertex-centric, two-level-parallel form of Alg. 2 (§3.3) over the paper's
 * compressed residual layouts RCSR and BCSR (§3.2, Fig. 2), with the global
 * relabel heuristic of §2.2 and the gap heuristic.
 *
 * Conventions for every call:
 *  - Vertices are 0 .. n-1.  Arcs are three int32 arrays src[m], dst[m],
 *    cap[m] with cap >= 0.  Self-loops are accepted and carry flow 0.  Parallel
 *    and antiparallel arcs are accepted.
 *  - Integer arithmetic throughout: residual capacities int32, excesses and
 *    flow values int64.  Results are exact.
 *  - A stream argument is a cudaStream_t (NULL = the legacy default stream).
 *    A handle must be used by one stream at a time; different handles are
 *    independent.
 *  - No call aborts, traps or prints.  Failures return a negative
 *    wbpr_status (or NULL from the build calls); wbpr_last_error() and
 *    wbpr_last_error_message() then describe the last failure of the calling
 *    thread.
 */
#ifndef WBPR_H
#define WBPR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *wbpr_stream_t; /* same type as cudaStream_t */
typedef struct wbpr_graph wbpr_graph;      /* opaque; owns all device memory of one instance */

/* Residual-graph layouts of §3.2 (Fig. 2(c), 2(d)). */
typedef enum {
    WBPR_RCSR = 0, /* out-arc CSR plus an in-arc CSR whose entries hold flow_idx,
                      the slot of the backward flow (constant-time backward access) */
    WBPR_BCSR = 1  /* one merged neighbour list per vertex sorted by neighbour id;
                      backward slot by binary search or a precomputed reverse index */
} wbpr_layout;

typedef enum {
    WBPR_OK = 0,
    WBPR_EINVAL = -1,    /* bad argument: n < 2, m < 0, s == t, id out of range,
                            negative capacity, bad layout, NULL required pointer */
    WBPR_ENOMEM = -2,    /* a device or host allocation failed */
    WBPR_ECUDA = -3,     /* a CUDA runtime call failed (no device, launch error...) */
    WBPR_ETIMEOUT = -4,  /* the iteration cap or a device wait limit was reached;
                            the handle stays usable (solve again or destroy) */
    WBPR_EOVERFLOW = -5, /* a vertex's capacity sum exceeds INT64_MAX, a merged
                            pair c(u,v)+c(v,u) exceeds INT32_MAX, n >= 2^30, or the
                            residual graph has 2^32 or more slots */
    WBPR_ESTATE = -6     /* misuse: e.g. a batch entry is NULL or repeated */
} wbpr_status;

/* Tuning knobs.  None of them changes a result; all of them change speed. */
typedef struct wbpr_options {
    int32_t use_rev;          /* BCSR backward-slot lookup: 1 = reverse index (default),
                                 0 = binary search in the neighbour's row (§3.2).
                                 Taken at build time: a handle built with 0 holds
                                 neither the reverse index nor the mirrored reverse
                                 residual (8 bytes per slot less) and refuses a
                                 later switch to 1 (WBPR_ESTATE) */
    int32_t gap;              /* 1 = gap heuristic on (default), 0 = off */
    int32_t multi_push;       /* 1 = discharge pass: the owner of u pushes along every
                                 arc read as lower in one pass, then relabels if excess
                                 is left (default); 0 = one push to the lowest
                                 neighbour or one relabel per iteration (Alg. 1, 2) */
    int32_t cycle;            /* push-relabel iterations between global relabels
                                 (the "cycle" of Alg. 1); 0 = automatic */
    int32_t small_max_degree; /* rows up to this length get a tile of
                                 `small_tile` lanes (default 8) */
    int32_t small_tile;       /* 4, 8 or 16 lanes (default 8) */
    int32_t warp_max_degree;  /* longer rows (up to this) get one warp; longer
                                 rows (hubs) are split into chunks of 2048 entries
                                 that whole thread blocks take (default 1024) */
    int32_t grid_blocks;      /* persistent grid size; 0 = automatic.  Clamped to
                                 the number of co-resident blocks.  For
                                 wbpr_maxflow_batch (options of the first handle)
                                 it caps the batch grid instead. */
    int32_t barrier_timeout_ms; /* device wait limit (default 20000) */
    int64_t max_iterations;   /* cap on push-relabel iterations per solve
                                 (default 2^40); reaching it gives WBPR_ETIMEOUT */
    int32_t trace;            /* > 0: record up to this many grid barriers of each
                                 solve (barrier id, queue generation, device time in ns,
                                 queue sizes); read with wbpr_export(WBPR_ARRAY_TRACE) */
    float gr_ratio;           /* > 0: start a global relabel once the push-relabel
                                 iterations since the last one took gr_ratio times
                                 as long as it did (default 1.5); `cycle` then only
                                 caps the iterations in between.  0 = every `cycle`
                                 iterations */
    int32_t batch_team;       /* wbpr_maxflow_batch: blocks that solve one large
                                 instance together (power of two, default 16) */
    int64_t batch_big_slots;  /* wbpr_maxflow_batch: instances with more residual
                                 slots than this are large (default 2^15); smaller
                                 ones are solved by a single block each */
    int32_t bottom_up;        /* BFS direction (global relabel and min cut).  A level whose
                                 frontier F has at least bottom_up_min vertices and
                                 whose residual-list entries times bottom_up reach
                                 those of the vertices not yet visited (or, with
                                 bottom_up_edges = 0, |F| * bottom_up >= the
                                 vertices not yet visited) runs bottom-up: every
                                 unvisited vertex looks for a residual arc into F
                                 and stops at the first.  Otherwise top-down.
                                 0 = always top-down.  Default 14 */
    int32_t bottom_up_min;    /* default 1024 */
    int32_t renumber;         /* vertex numbering of the solver, fixed at build time:
                                 1 = renumber by endpoint count, largest first
                                 (the heights that residual scans gather from
                                 share cache sectors), 0 = input ids, -1 = automatic
                                 (default: on from 2^22 vertices).  Results are in
                                 input ids either way. */
    int32_t thread_centric;   /* 1 = the thread-centric baseline of §2.2 / §4 (TC):
                                 every thread owns fixed vertices, checks them for
                                 activity itself and scans an active vertex's whole
                                 residual list alone; no active-vertex queue, no
                                 degree classes.  0 = vertex-centric (default). */
    int32_t warp_time;        /* 1 = record, per warp of the grid, the device time
                                 spent in push-relabel passes (taken by the warp's
                                 first lane, summed over the solve); read with
                                 wbpr_export(WBPR_ARRAY_WARP_TIME).  Default 0. */
    int32_t stage_hubs;       /* 1 = stage the residual-list chunks of hub rows in shared
                                 memory: a warp copies its next chunk (cp.async) while
                                 it works on the current one (BCSR; 32 KB of shared
                                 memory per block).  0 = read them directly (default:
                                 the 4 x 49 KB of shared memory per SM leave the
                                 global-relabel BFS too little L1). */
    int32_t barrier_extra;    /* for tests of the device wait limit only: every grid
                                 barrier waits for this many arrivals more than the
                                 grid has, so its wait runs out after
                                 barrier_timeout_ms and the solve returns
                                 WBPR_ETIMEOUT (0..1024, default 0; grids of one
                                 block do not wait) */
    int32_t bottom_up_edges;  /* BFS direction rule: 1 = compare the residual-list
                                 entries of the frontier, times bottom_up, with
                                 those of the vertices not yet visited; 0 = compare
                                 vertex counts; 2 = entries in the global relabels
                                 of phase 1 and in the cut, vertex counts in the
                                 global relabels of phase 2; -1 = automatic (default):
                                 2 from 2^21 vertices, else 0 */
    int32_t avq_incremental;  /* 1 = between two global relabels, build the AVQ only
                                 from the vertices the last pass pushed into or left
                                 with excess (a bitmap the pushes mark); the first
                                 compaction after a global relabel, and one that
                                 applies a gap, scan every vertex.  2 = as 1, and
                                 while the AVQ stays small (at most 64 vertices per
                                 block, no hub) every block compacts and processes
                                 the marked vertices of its own bitmap words in the
                                 same pass, saving a grid barrier per iteration
                                 (default).  0 = every compaction scans every
                                 vertex (Alg. 2). */
    int32_t lean_build;       /* build time: 1 = every block the builder launches fits
                                 beside two blocks of a resident server kernel per SM
                                 (radix sorts with 256-thread blocks, duplicate-arc
                                 prefixes by run; never renumbers), for builds that
                                 run while wbpr_server_start's kernel is resident.
                                 0 = CUB's own tuning (default, faster alone). */
} wbpr_options;

/* Counters of the last solve on a handle. */
typedef struct wbpr_stats {
    int64_t iterations;        /* push-relabel iterations (Alg. 2 passes), both phases */
    int64_t phase1_iterations;
    int64_t global_relabels;   /* backward BFS passes, both phases */
    int64_t active_total;      /* sum over iterations of |AVQ| */
    int64_t arcs_scanned;      /* residual-list entries read by the min-height scans */
    int64_t gr_arcs_scanned;   /* entries read by the global-relabel BFS */
    int64_t pushes;
    int64_t relabels;
    int64_t gaps;              /* gap-heuristic liftings applied */
    int64_t written_off;       /* excess written off by global relabels (§2.2) */
    double  solve_ms;          /* device time of the last wbpr_maxflow/_mincut solve */
    int64_t avq_full_scans;    /* AVQ compactions that scanned every vertex */
    int64_t avq_bitmap_scans;  /* AVQ compactions from the candidate bitmap (avq_incremental) */
    int64_t avq_candidates;    /* marked vertices those compactions examined */
} wbpr_stats;

/* Sizes of a built handle. */
typedef struct wbpr_info {
    int64_t n, m;              /* as given to wbpr_build */
    int32_t s, t;
    int32_t layout;            /* wbpr_layout */
    int64_t slots;             /* BCSR: merged neighbour entries (2 x unordered pairs);
                                  RCSR: out-arcs (= in-arcs) without self-loops */
    int64_t max_degree;        /* longest residual list */
    int64_t device_bytes;      /* device memory held by the handle */
    int32_t grid_blocks;       /* persistent grid used by the solver */
    int32_t num_sms;
    int32_t renumbered;        /* 1 when the solver numbers vertices differently
                                  from the input (wbpr_options.renumber) */
} wbpr_info;

/*
 * wbpr_build -- build the residual graph of §3.2 in the chosen layout.
 *   n, m        vertex and arc counts (n >= 2, m >= 0, n < 2^30, m < 2^31).
 *   src,dst,cap arc arrays of m int32 each; host or device pointers (detected
 *               per pointer).  Read during the call only; the caller keeps them.
 *   s, t        source and sink (0 <= s, t < n, s != t).
 *   layout      WBPR_RCSR or WBPR_BCSR.
 * Runs on the legacy default stream and returns after the graph is built.
 * Returns a handle owning all device memory of the instance, or NULL on error
 * (see wbpr_last_error()).
 */
wbpr_graph *wbpr_build(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                       const int32_t *cap, int32_t s, int32_t t, wbpr_layout layout);

/* Same as wbpr_build, on `stream`, with options (NULL = defaults). */
wbpr_graph *wbpr_build_ex(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                          const int32_t *cap, int32_t s, int32_t t, wbpr_layout layout,
                          const wbpr_options *opts, wbpr_stream_t stream);

/*
 * wbpr_maxflow -- solve for a maximum flow (Alg. 1 driven by Alg. 2).
 *   value      host pointer, required: receives the maximum flow value e(t).
 *   edge_flow  NULL, or m int32 (host or device pointer): receives the flow on
 *              every input arc in input order.  When non-NULL a second phase
 *              returns stranded excess to s so the flow is valid: 0 <= f <= cap,
 *              conservation at every vertex other than s and t.  Parallel arcs
 *              share their pair's flow greedily in input order; a self-loop
 *              gets 0.  A page-locked host buffer that is mapped into the
 *              device's address space (pinned memory on a system with
 *              unified addressing) is written directly by the kernel that
 *              computes the flows; other host buffers are staged in device
 *              memory and copied.
 * Re-solves from scratch on every call (idempotent).  Synchronises `stream`
 * before returning.
 */
wbpr_status wbpr_maxflow(wbpr_graph *g, wbpr_stream_t stream, int64_t *value,
                         int32_t *edge_flow);

/*
 * wbpr_maxflow_async -- as wbpr_maxflow but stream-ordered with no host
 * synchronisation and no allocation: d_value (device int64, required) and
 * d_edge_flow (device int32[m] or NULL) are written in stream order.  The
 * status of the solve is read later by wbpr_solve_status().  The handle's
 * own buffers are reused, so overlapping calls on one handle race.
 */
wbpr_status wbpr_maxflow_async(wbpr_graph *g, wbpr_stream_t stream, int64_t *d_value,
                               int32_t *d_edge_flow);

/* Device-side status of the last stream-ordered solve (synchronises `stream`). */
wbpr_status wbpr_solve_status(wbpr_graph *g, wbpr_stream_t stream);

/*
 * wbpr_mincut -- a minimum s-t cut (max-flow = min-cut, §1).
 *   cut_value   host pointer, required: the cut capacity (= the max-flow value).
 *   source_side NULL, or n bytes (host or device pointer): 1 for the vertices
 *               reachable from s in the residual graph of a maximum flow (the
 *               smallest minimum-cut source side; the same for every maximum
 *               flow), else 0.  Mapped page-locked host buffers are
 *               written directly, as for wbpr_maxflow's edge flows.
 * Reuses the state of a previous wbpr_maxflow with edge flows on this handle;
 * otherwise solves first.  Synchronises `stream`.
 */
wbpr_status wbpr_mincut(wbpr_graph *g, wbpr_stream_t stream, int64_t *cut_value,
                        uint8_t *source_side);

/*
 * wbpr_maxflow_batch -- solve `count` independent instances in one launch.
 *   gs          count distinct handles (all built on this device).
 *   values      host int64[count], required.
 *   edge_flows  NULL, or count pointers each NULL or an int32[m_i] device
 *               buffer for instance i.
 * Each result equals that of wbpr_maxflow on the same handle.
 */
wbpr_status wbpr_maxflow_batch(wbpr_graph *const *gs, int32_t count, wbpr_stream_t stream,
                               int64_t *values, int32_t *const *edge_flows);

/* Release every device buffer of the handle.  NULL is accepted.  No work of
 * the handle may be in flight (synchronise after wbpr_maxflow_async). */
void wbpr_destroy(wbpr_graph *g);

/* Options: defaults, read, replace (takes effect at the next solve). */
void wbpr_default_options(wbpr_options *opts);
wbpr_status wbpr_get_options(const wbpr_graph *g, wbpr_options *opts);
wbpr_status wbpr_set_options(wbpr_graph *g, const wbpr_options *opts);

/* Counters of the last solve; sizes of the handle. */
wbpr_status wbpr_get_stats(const wbpr_graph *g, wbpr_stats *stats);
wbpr_status wbpr_get_info(const wbpr_graph *g, wbpr_info *info);

/* Last failure of the calling thread; a static description of a status. */
wbpr_status wbpr_last_error(void);
const char *wbpr_last_error_message(void);
const char *wbpr_error_string(wbpr_status status);

/*
 * Device allocator hook.  By default the library allocates with
 * cudaMallocAsync/cudaFreeAsync on the call's stream.  A host framework can
 * route every device allocation of later calls through its own allocator
 * (for example PyTorch's caching allocator).  alloc returns NULL on failure.
 * Pass NULL functions to restore the default.  Not thread-safe against
 * concurrent library calls.
 */
typedef void *(*wbpr_alloc_fn)(size_t bytes, wbpr_stream_t stream, void *ctx);
typedef void (*wbpr_free_fn)(void *ptr, size_t bytes, wbpr_stream_t stream, void *ctx);
wbpr_status wbpr_set_allocator(wbpr_alloc_fn alloc, wbpr_free_fn free_fn, void *ctx);

/*
 * Stage-level access for testing each step of the method on its own.
 *   wbpr_run_stage(g, stream, stage, arg):
 *     WBPR_STAGE_PREFLOW          reset to the initial residual graph, then the
 *                                 preflow of Alg. 1 step 0 (h(s)=n, others 0)
 *     WBPR_STAGE_GLOBAL_RELABEL   one global relabel of §2.2 on the current
 *                                 state (backward BFS from t, write-off)
 *     WBPR_STAGE_ITERATIONS       `arg` push-relabel iterations of Alg. 2 on
 *                                 the current state, without global relabel
 *   wbpr_export(g, what, host_dst, count): copy `count` elements of an
 *     internal array to host memory (synchronous).  Per-vertex arrays and the
 *     layout are in the solver's vertex numbering: the input ids, unless the
 *     handle was renumbered (wbpr_options.renumber), in which case
 *     WBPR_ARRAY_ORDER maps each solver id to its input id and WBPR_ARRAY_ST
 *     gives the solver ids of s and t.
 */
enum {
    WBPR_STAGE_PREFLOW = 1,
    WBPR_STAGE_GLOBAL_RELABEL = 2,
    WBPR_STAGE_ITERATIONS = 3
};
enum {
    WBPR_ARRAY_HEIGHT = 1,      /* int32[n] */
    WBPR_ARRAY_EXCESS = 2,      /* int64[n] */
    WBPR_ARRAY_OFFSETS = 3,     /* int64[n+1]: BCSR rows / RCSR out rows */
    WBPR_ARRAY_COL = 4,         /* int32[slots]: neighbour of each slot */
    WBPR_ARRAY_CF = 5,          /* int32[slots]: residual capacity of each slot
                                   (RCSR: of the forward arc) */
    WBPR_ARRAY_CAP = 6,         /* int32[slots]: initial residual capacity */
    WBPR_ARRAY_REV = 7,         /* uint32[slots]: BCSR reverse slot */
    WBPR_ARRAY_BF = 8,          /* int32[slots]: RCSR backward residual (flow) */
    WBPR_ARRAY_IN_OFFSETS = 9,  /* int64[n+1]: RCSR in rows */
    WBPR_ARRAY_IN_COL = 10,     /* int32[slots]: RCSR in-arc tail */
    WBPR_ARRAY_FLOW_IDX = 11,   /* uint32[slots]: RCSR in-arc -> out slot */
    WBPR_ARRAY_ARC2SLOT = 12,   /* uint32[m]: input arc -> slot (UINT32_MAX for loops) */
    WBPR_ARRAY_EXCESS_TOTAL = 13, /* int64[1] */
    WBPR_ARRAY_TRACE = 14,       /* uint64[4 * records]: per grid barrier of the last
                                    launch: barrier id, queue generation, globaltimer ns,
                                    queue sizes (24 bits per tile class) */
    WBPR_ARRAY_TRACE_LEN = 15,   /* uint32[1]: records in the trace */
    WBPR_ARRAY_ORDER = 16,       /* int32[n]: input id of each solver vertex id
                                    (0 elements when the handle is not renumbered) */
    WBPR_ARRAY_ST = 17,          /* int32[2]: solver ids of s and t (host copy) */
    WBPR_ARRAY_WARP_TIME = 18    /* uint64[grid_blocks * 8]: per warp of the last
                                    launch's grid, ns spent in push-relabel passes
                                    (wbpr_options.warp_time; 0 elements when off) */
};
wbpr_status wbpr_run_stage(wbpr_graph *g, wbpr_stream_t stream, int32_t stage, int64_t arg);
wbpr_status wbpr_export(const wbpr_graph *g, int32_t what, void *host_dst, int64_t count);

/*
 * wbpr_maxflow_bcsr_noalloc -- maximum flow value of a small graph that the
 * caller already holds in the BCSR layout, without allocating any memory.
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory while they run -- code inside a host framework's
 * execution phase that forbids allocation (a plugin's enqueue step, say),
 * real-time loops whose device memory budget is fixed up front, or embedders
 * that own no CUDA allocator.  It calls no cudaMalloc, cudaFree or allocating
 * library routine: the solver's working set (residual capacities, excesses,
 * heights, queues, control block) lives in one fixed device array of about
 * 15.6 MiB that every GPU loading the library holds until the process exits.
 *   n, slots   vertex count (2 .. WBPR_NOALLOC_MAX_VERTICES) and BCSR entry
 *              count (0 .. WBPR_NOALLOC_MAX_SLOTS); larger graphs are rejected
 *              with WBPR_EINVAL.
 *   s, t       source and sink.
 *   off, col, cap, rev  device arrays of the BCSR layout (as wbpr_export
 *              returns them for WBPR_ARRAY_OFFSETS, _COL, _CAP, _REV): int64
 *              row offsets [n+1], int32 neighbour ids [slots] sorted within
 *              each row, int32 initial residual capacities [slots], uint32
 *              paired slot of each entry [slots].  Read only.
 *   d_value    device int64: receives the maximum flow value.
 *   d_residual NULL, or device int32[slots]: receives the residual capacity
 *              of every slot at the end of the solve (cap - residual is the
 *              flow of a maximum preflow).
 * Before solving, a kernel checks the arrays: off[0] = 0, off[n] = slots, rows
 * non-decreasing, neighbour ids in [0, n), capacities >= 0, and rev[] pairing
 * every slot with one in its neighbour's row that points back.  Arrays that
 * fail return WBPR_EINVAL and nothing is solved.  The call synchronises
 * `stream` (twice: after the check and after the solve) and returns the
 * solve's status; because it synchronises, no call of it can be recorded
 * into a CUDA graph by stream capture.  The first call on a device looks up
 * the array's device address (once per device, with that device current).  Every
 * call shares the one array, which keeps the last call's contents (the call
 * clears what must start at zero), so calls that overlap on the GPU -- from
 * two host threads or two streams -- race and must not be issued.
 */
#define WBPR_NOALLOC_MAX_VERTICES 65536
#define WBPR_NOALLOC_MAX_SLOTS 1048576
wbpr_status wbpr_maxflow_bcsr_noalloc(int32_t n, int64_t slots, int32_t s, int32_t t,
                                      const int64_t *off, const int32_t *col, const int32_t *cap,
                                      const uint32_t *rev, wbpr_stream_t stream, int64_t *d_value,
                                      int32_t *d_residual);

/*
 * Persistent server (continuous batching).  wbpr_server_start launches one
 * long-running kernel on its own non-blocking stream.  Its blocks form
 * `big_teams` teams of `team_blocks` blocks for large instances and
 * `small_blocks` single-block teams for small ones.  wbpr_server_submit
 * publishes a built handle to the queue of its size class (more than
 * `big_slots` residual slots = large); the first free team of that class
 * solves it at once, while other requests are being solved.  The call does
 * not block.  wbpr_server_poll returns WBPR_OK with the flow value once the
 * request is done, or 1 while it is pending (WBPR_ESTATE if the kernel has
 * exited without solving it).  A handle must not be used in
 * any other call between its submit and the poll that reports it done.
 * wbpr_server_stop lets the running solves finish, stops the kernel (which
 * also stops on its own after `idle_ms` without requests), and frees the
 * server.  `idle_ms` (default 60 s) is only a safety net for a host that
 * stopped submitting without calling wbpr_server_stop: a team that waited
 * that long for its next request leaves the kernel, and a request published
 * to its queue position afterwards is never solved (its poll then reports
 * WBPR_ESTATE).  The rings hold `capacity` requests per class for the lifetime of
 * the server.  Only handles with the server's layout are accepted.
 * Host-mapped pinned memory carries requests and results (no device
 * round trip per request).  Leave room on the SMs: a build launched while
 * the server runs needs resident space for its own blocks, and it waits for
 * the server to exit otherwise.  Its radix-sort blocks need about 37 K
 * registers, more than an SM holding two server blocks (16 K each) has left,
 * so the defaults use one server block per SM (4 teams of 16 blocks and 88
 * single-block teams on 152 SMs).  wbpr_maxflow_batch builds nothing while
 * its server runs and uses every resident slot.
 */
typedef struct wbpr_server wbpr_server;
typedef struct wbpr_server_options {
    int32_t layout;        /* WBPR_RCSR or WBPR_BCSR */
    int32_t capacity;      /* requests per class over the server's lifetime */
    int32_t team_blocks;   /* blocks per large-instance team (power of two) */
    int32_t big_teams;     /* large-instance teams */
    int32_t small_blocks;  /* single-block teams */
    int32_t idle_ms;       /* the kernel stops after this long without requests */
    int64_t big_slots;     /* class boundary in residual slots */
    int32_t build_room;    /* 1 = the server kernel asks for the largest shared-memory
                              carveout, so that the blocks of builds that run while it
                              is resident (lean builds, wbpr_options.lean_build) find
                              shared memory beside two server blocks per SM (default);
                              0 = the default carveout (more L1; nothing is built
                              while the server runs) */
} wbpr_server_options;
void wbpr_server_default_options(wbpr_server_options *opts);
wbpr_server *wbpr_server_start(const wbpr_server_options *opts);
int64_t wbpr_server_submit(wbpr_server *srv, wbpr_graph *g);  /* ticket >= 0, or a negative wbpr_status */
wbpr_status wbpr_server_poll(wbpr_server *srv, int64_t ticket, int64_t *value);
wbpr_status wbpr_server_stop(wbpr_server *srv);
/* Device interval of a finished request: the server kernel's globaltimer (ns)
 * when its team started and finished the solve.  WBPR_OK once the request is
 * done (as wbpr_server_poll reports), 1 while it is pending.  The values stay
 * readable until wbpr_server_stop. */
wbpr_status wbpr_server_times(wbpr_server *srv, int64_t ticket, uint64_t *t_start_ns, uint64_t *t_end_ns);
/* Diagnostics once the server kernel has ended (1 while it still runs): for
 * each of the first `count` teams (large teams first, then single blocks) why
 * it left: 0 still running, 1 end of its ring, 2 stop flag, 3 idle limit,
 * 4-6 a team barrier gave up. */
wbpr_status wbpr_server_team_exits(wbpr_server *srv, int32_t *reasons, int32_t count);

#ifdef __cplusplus
}
#endif
#endif /* WBPR_H */
