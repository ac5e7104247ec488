// C ABI of the WBPR library: argument checks, handle lifecycle, device
// allocation (through the allocator hook), and the host side of each solve.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "handle.h"
#include "wbpr.h"

namespace wbpr {
namespace {

thread_local wbpr_status t_last = WBPR_OK;
thread_local std::string t_msg;

wbpr_alloc_fn g_alloc = nullptr;
wbpr_free_fn g_free = nullptr;
void *g_ctx = nullptr;

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The device address of a page-locked host buffer that kernels can write
// directly (mapped into the device's address space), else null.  Outputs
// in such buffers are written by the kernel that computes them, over the
// host link, instead of being staged in device memory and copied.
void *mapped_host_ptr(void *p)
{
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

}  // namespace

wbpr_status set_error(wbpr_status st, const std::string &msg)
{
    t_last = st;
    t_msg = msg;
    return st;
}

void *dev_alloc(size_t bytes, cudaStream_t stream, DevFree *owner)
{
    if (owner) *owner = DevFree{g_free, g_ctx};
    if (g_alloc) return g_alloc(bytes, (wbpr_stream_t)stream, g_ctx);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void *p, size_t bytes, cudaStream_t stream, const DevFree *owner)
{
    if (!p) return;
    const wbpr_free_fn fn = owner ? owner->fn : g_free;
    void *ctx = owner ? owner->ctx : g_ctx;
    if (fn) {
        fn(p, bytes, (wbpr_stream_t)stream, ctx);
        return;
    }
    cudaFreeAsync(p, stream);
}

}  // namespace wbpr

using namespace wbpr;

#define API_CUDA(call)                                                                  \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return set_error(WBPR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

extern "C" {

void wbpr_default_options(wbpr_options *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->use_rev = 1;
    o->gap = 1;
    o->multi_push = 1;
    o->cycle = 0;
    o->small_max_degree = 8;
    o->small_tile = 8;
    o->warp_max_degree = 1024;
    o->grid_blocks = 0;
    o->barrier_timeout_ms = 20000;
    o->max_iterations = (int64_t)1 << 40;
    o->trace = 0;
    o->gr_ratio = 1.5f;
    o->batch_team = 16;
    o->batch_big_slots = (int64_t)1 << 15;
    o->bottom_up = 14;
    o->bottom_up_min = 1024;
    o->renumber = -1;
    o->thread_centric = 0;
    o->warp_time = 0;
    o->stage_hubs = 0;
    o->barrier_extra = 0;
    o->bottom_up_edges = -1;
    o->avq_incremental = 2;
}

wbpr_status wbpr_last_error(void) { return t_last; }

const char *wbpr_last_error_message(void) { return t_msg.c_str(); }

const char *wbpr_error_string(wbpr_status st)
{
    switch (st) {
    case WBPR_OK: return "success";
    case WBPR_EINVAL: return "invalid argument";
    case WBPR_ENOMEM: return "out of memory";
    case WBPR_ECUDA: return "CUDA error";
    case WBPR_ETIMEOUT: return "iteration cap or device wait limit reached";
    case WBPR_EOVERFLOW: return "capacity or size overflow";
    case WBPR_ESTATE: return "invalid state or misuse";
    }
    return "unknown status";
}

wbpr_status wbpr_set_allocator(wbpr_alloc_fn alloc, wbpr_free_fn free_fn, void *ctx)
{
    if ((alloc == nullptr) != (free_fn == nullptr))
        return set_error(WBPR_EINVAL, "wbpr_set_allocator: give both functions or neither");
    g_alloc = alloc;
    g_free = free_fn;
    g_ctx = ctx;
    return WBPR_OK;
}

static wbpr_status check_options(const wbpr_options *o)
{
    if (o->use_rev != 0 && o->use_rev != 1) return WBPR_EINVAL;
    if (o->gap != 0 && o->gap != 1) return WBPR_EINVAL;
    if (o->multi_push != 0 && o->multi_push != 1) return WBPR_EINVAL;
    if (o->cycle < 0) return WBPR_EINVAL;
    if (o->small_tile != 4 && o->small_tile != 8 && o->small_tile != 16) return WBPR_EINVAL;
    if (o->small_max_degree < 0 || o->warp_max_degree < o->small_max_degree) return WBPR_EINVAL;
    if (o->grid_blocks < 0 || o->barrier_timeout_ms <= 0 || o->max_iterations <= 0) return WBPR_EINVAL;
    if (o->trace < 0 || o->trace > (1 << 24)) return WBPR_EINVAL;
    if (!(o->gr_ratio >= 0.f && o->gr_ratio < 1e6f)) return WBPR_EINVAL;
    if (o->batch_team < 1 || o->batch_team > 64 || (o->batch_team & (o->batch_team - 1))) return WBPR_EINVAL;
    if (o->batch_big_slots < 0) return WBPR_EINVAL;
    if (o->bottom_up < 0 || o->bottom_up > (1 << 20) || o->bottom_up_min < 1) return WBPR_EINVAL;
    if (o->renumber < -1 || o->renumber > 1) return WBPR_EINVAL;
    if (o->thread_centric != 0 && o->thread_centric != 1) return WBPR_EINVAL;
    if (o->warp_time != 0 && o->warp_time != 1) return WBPR_EINVAL;
    if (o->barrier_extra < 0 || o->barrier_extra > 1024) return WBPR_EINVAL;
    if (o->stage_hubs != 0 && o->stage_hubs != 1) return WBPR_EINVAL;
    if (o->bottom_up_edges < -1 || o->bottom_up_edges > 2) return WBPR_EINVAL;
    if (o->avq_incremental < 0 || o->avq_incremental > 2) return WBPR_EINVAL;
    if (o->lean_build != 0 && o->lean_build != 1) return WBPR_EINVAL;
    return WBPR_OK;
}

void wbpr_destroy(wbpr_graph *g)
{
    if (!g) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(g->device);
    // Not a device-wide sync: a persistent server kernel may be running on a
    // non-blocking stream.  The caller guarantees no work of this handle is in
    // flight (every synchronous call has finished it).
    cudaStreamSynchronize(0);
    for (auto &b : g->blocks) dev_free(b.p, b.bytes, 0, &b.owner);
    cudaStreamSynchronize(0);
    delete[] g->pinned;
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    cudaGetLastError();
    cudaSetDevice(prev);
    delete g;
}

static wbpr_status alloc_state(wbpr_graph *g, cudaStream_t st)
{
    const int64_t n = g->n;
#define STATE_ALLOC(ptr, type, count)                                              \
    do {                                                                           \
        ptr = (type *)g->alloc(sizeof(type) * (size_t)(count), st);                \
        if (!ptr) return set_error(WBPR_ENOMEM, "state: device allocation failed"); \
    } while (0)
    STATE_ALLOC(g->e, long long, n);
    STATE_ALLOC(g->h, int, n);
    STATE_ALLOC(g->dead, unsigned char, n);
    STATE_ALLOC(g->count, int, n + 1);
    for (int a = 0; a < 2; ++a) {
        for (int k = 0; k < kClasses; ++k) STATE_ALLOC(g->q[a][k], int, n);
        STATE_ALLOC(g->hub_start[a], unsigned, n);
        STATE_ALLOC(g->hub_chunk[a], unsigned,
                    hub_chunk_entries(n, g->slots, g->layout == WBPR_BCSR ? kBCSR : kRCSR));
        STATE_ALLOC(g->hub_e0[a], long long, n);
        STATE_ALLOC(g->hub_rem[a], long long, n);
        STATE_ALLOC(g->hub_aux[a], unsigned long long, n);
        STATE_ALLOC(g->hub_done[a], unsigned, n);
    }
    STATE_ALLOC(g->touch, unsigned, (n + 31) / 32);
    STATE_ALLOC(g->ctl, Ctl, 1);
    int per_sm = 0;
    API_CUDA(solver_max_blocks_per_sm(g->layout, 8, &per_sm));
    int per_sm4 = 0, per_sm16 = 0;
    API_CUDA(solver_max_blocks_per_sm(g->layout, 4, &per_sm4));
    API_CUDA(solver_max_blocks_per_sm(g->layout, 16, &per_sm16));
    per_sm = std::max(per_sm, std::max(per_sm4, per_sm16));
    g->bstats_blocks = std::max(1, per_sm) * g->num_sms;
    STATE_ALLOC(g->bstats, long long, (int64_t)g->bstats_blocks * kStatCount);
#undef STATE_ALLOC
    return WBPR_OK;
}

wbpr_graph *wbpr_build_ex(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                          const int32_t *cap, int32_t s, int32_t t, wbpr_layout layout,
                          const wbpr_options *opts, wbpr_stream_t stream)
{
    if (n < 2 || m < 0 || s < 0 || t < 0 || s >= n || t >= n || s == t) {
        set_error(WBPR_EINVAL, "wbpr_build: need n >= 2, m >= 0, 0 <= s,t < n, s != t");
        return nullptr;
    }
    if (n >= ((int64_t)1 << 30) || m >= ((int64_t)1 << 31)) {
        set_error(WBPR_EOVERFLOW, "wbpr_build: n must be below 2^30 and m below 2^31");
        return nullptr;
    }
    if (layout != WBPR_RCSR && layout != WBPR_BCSR) {
        set_error(WBPR_EINVAL, "wbpr_build: unknown layout");
        return nullptr;
    }
    if (m > 0 && (!src || !dst || !cap)) {
        set_error(WBPR_EINVAL, "wbpr_build: NULL arc array");
        return nullptr;
    }
    wbpr_options o;
    wbpr_default_options(&o);
    if (opts) o = *opts;
    if (check_options(&o) != WBPR_OK) {
        set_error(WBPR_EINVAL, "wbpr_build: invalid options");
        return nullptr;
    }
    cudaStream_t st = (cudaStream_t)stream;
    wbpr_graph *g = new wbpr_graph();
    g->n = n;
    g->m = m;
    g->s = s;
    g->t = t;
    g->layout = layout;
    g->opts = o;
    g->lean = o.lean_build != 0;
    // (a lean build never renumbers: the renumbering sort runs on CUB's own tuning)
    g->renumbered = !g->lean && (o.renumber == 1 || (o.renumber == -1 && n >= kRenumberAutoVertices));
    memset(&g->stats, 0, sizeof(g->stats));
    auto fail = [&](wbpr_status code, const std::string &msg) -> wbpr_graph * {
        wbpr_status keep = t_last == WBPR_OK ? code : t_last;
        std::string keep_msg = t_msg.empty() ? msg : t_msg;
        wbpr_destroy(g);
        set_error(keep, keep_msg);
        return nullptr;
    };
    t_last = WBPR_OK;
    t_msg.clear();
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        cudaGetLastError();
        delete g;
        set_error(WBPR_ECUDA, "wbpr_build: no CUDA device");
        return nullptr;
    }
    cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, g->device);
    if (!coop) return fail(WBPR_ECUDA, "wbpr_build: device lacks cooperative launch");
    // Host staging of small results: ordinary heap memory.  A pinned
    // allocation here would synchronise with every stream (including a
    // running persistent server kernel).
    g->pinned = new (std::nothrow) long long[64];
    if (!g->pinned) {
        return fail(WBPR_ENOMEM, "wbpr_build: host allocation failed");
    }
    cudaEventCreate(&g->ev0);
    cudaEventCreate(&g->ev1);
    // Inputs on the host are staged to the device for the duration of the build.
    const int32_t *arr[3] = {src, dst, cap};
    const int32_t *dev_arr[3] = {src, dst, cap};
    void *staged[3] = {nullptr, nullptr, nullptr};
    const size_t bytes = sizeof(int32_t) * (size_t)(m > 0 ? m : 1);
    for (int k = 0; k < 3 && m > 0; ++k) {
        if (!is_device_ptr(arr[k])) {
            staged[k] = dev_alloc(bytes, st);
            if (!staged[k]) {
                for (int j = 0; j < k; ++j) dev_free(staged[j], bytes, st);
                return fail(WBPR_ENOMEM, "wbpr_build: staging allocation failed");
            }
            if (cudaMemcpyAsync(staged[k], arr[k], bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
                cudaGetLastError();
                for (int j = 0; j <= k; ++j) dev_free(staged[j], bytes, st);
                return fail(WBPR_ECUDA, "wbpr_build: host-to-device copy failed");
            }
            dev_arr[k] = (const int32_t *)staged[k];
        }
    }
    wbpr_status rc = build_graph(g, dev_arr[0], dev_arr[1], dev_arr[2], st);
    for (int k = 0; k < 3; ++k)
        if (staged[k]) dev_free(staged[k], bytes, st);
    if (rc != WBPR_OK) return fail(rc, "wbpr_build failed");
    if (g->slots >= ((int64_t)1 << 32) - 1) return fail(WBPR_EOVERFLOW, "wbpr_build: 2^32 or more slots");
    rc = alloc_state(g, st);
    if (rc != WBPR_OK) return fail(rc, "wbpr_build: state allocation failed");
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        std::string msg = std::string("wbpr_build: ") + cudaGetErrorString(cudaGetLastError());
        return fail(WBPR_ECUDA, msg);
    }
    return g;
}

wbpr_graph *wbpr_build(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                       const int32_t *cap, int32_t s, int32_t t, wbpr_layout layout)
{
    return wbpr_build_ex(n, m, src, dst, cap, s, t, layout, nullptr, nullptr);
}

wbpr_status wbpr_get_options(const wbpr_graph *g, wbpr_options *o)
{
    if (!g || !o) return set_error(WBPR_EINVAL, "wbpr_get_options: NULL argument");
    *o = g->opts;
    return WBPR_OK;
}

wbpr_status wbpr_set_options(wbpr_graph *g, const wbpr_options *o)
{
    if (!g || !o) return set_error(WBPR_EINVAL, "wbpr_set_options: NULL argument");
    if (check_options(o) != WBPR_OK) return set_error(WBPR_EINVAL, "wbpr_set_options: invalid options");
    if (o->renumber != g->opts.renumber)
        return set_error(WBPR_ESTATE, "wbpr_set_options: renumber is fixed when the handle is built");
    if (g->layout == WBPR_BCSR && o->use_rev && !g->rev)
        return set_error(WBPR_ESTATE, "wbpr_set_options: the handle was built without the reverse index (use_rev = 0)");
    g->opts = *o;
    return WBPR_OK;
}

wbpr_status wbpr_get_stats(const wbpr_graph *g, wbpr_stats *s)
{
    if (!g || !s) return set_error(WBPR_EINVAL, "wbpr_get_stats: NULL argument");
    *s = g->stats;
    return WBPR_OK;
}

wbpr_status wbpr_get_info(const wbpr_graph *g, wbpr_info *info)
{
    if (!g || !info) return set_error(WBPR_EINVAL, "wbpr_get_info: NULL argument");
    memset(info, 0, sizeof(*info));
    info->n = g->n;
    info->m = g->m;
    info->s = g->s;
    info->t = g->t;
    info->layout = g->layout;
    info->slots = g->slots;
    info->max_degree = g->max_degree;
    info->device_bytes = g->device_bytes;
    info->grid_blocks = g->grid_blocks;
    info->num_sms = g->num_sms;
    info->renumbered = g->order != nullptr;
    return WBPR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Solve orchestration
// ---------------------------------------------------------------------------
namespace wbpr {

static int auto_cycle(const wbpr_graph *g)
{
    // With the time-balanced trigger the cycle is only a cap.
    return g->opts.gr_ratio > 0.f ? 1000 : 16;
}

// Dynamic shared memory of a solver launch: the hub-chunk stage (BCSR).
static size_t launch_smem(const wbpr_graph *g)
{
    return g->opts.stage_hubs && g->layout == WBPR_BCSR ? (size_t)kStageBytes : 0;
}

static int choose_grid(wbpr_graph *g)
{
    int per_sm = 0;
    if (solver_max_blocks_per_sm(g->layout, g->opts.small_tile, &per_sm, launch_smem(g)) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    int maxg = per_sm * g->num_sms;
    if (maxg > g->bstats_blocks) maxg = g->bstats_blocks;
    int grid = g->opts.grid_blocks;
    if (grid <= 0) {
        // enough blocks to cover the vertex scan and the widest tiles, at most all co-resident
        long long want = (g->n + 4LL * kBlock - 1) / (4LL * kBlock);
        if (want < g->num_sms) want = g->num_sms;
        grid = (int)std::min<long long>(want, maxg);
    }
    if (grid > maxg) grid = maxg;
    if (grid < 1) grid = 1;
    return grid;
}

Params make_params(wbpr_graph *g, int mode)
{
    Params p;
    memset(&p, 0, sizeof(p));
    p.g.n = (int)g->n;
    p.g.s = g->s_int;
    p.g.t = g->t_int;
    p.g.order = g->order;
    p.g.perm = g->perm;
    p.g.slots = g->slots;
    p.g.off = g->off;
    p.g.col = g->col;
    p.g.cf = g->cf;
    p.g.cf0 = g->cf0;
    p.g.rev = g->rev;
    p.g.cfb = (g->layout == WBPR_BCSR && g->opts.use_rev) ? g->cfb : nullptr;
    p.g.bf = g->bf;
    p.g.in_off = g->in_off;
    p.g.in_col = g->in_col;
    p.g.flow_idx = g->flow_idx;
    p.st.e = g->e;
    p.st.h = g->h;
    p.st.dead = g->dead;
    p.st.count = g->count;
    for (int a = 0; a < 2; ++a) {
        for (int k = 0; k < kClasses; ++k) p.st.q[a][k] = g->q[a][k];
        p.st.hub_start[a] = g->hub_start[a];
        p.st.hub_chunk[a] = g->hub_chunk[a];
        p.st.hub_e0[a] = g->hub_e0[a];
        p.st.hub_rem[a] = g->hub_rem[a];
        p.st.hub_aux[a] = g->hub_aux[a];
        p.st.hub_done[a] = g->hub_done[a];
    }
    // (the thread-centric baseline builds no AVQ: its pushes mark nothing)
    p.st.touch = (g->opts.avq_incremental && !g->opts.thread_centric) ? g->touch : nullptr;
    p.local_passes = g->opts.avq_incremental >= 2 ? 1 : 0;
    p.st.ctl = g->ctl;
    p.st.bstats = g->bstats;
    p.mode = mode;
    p.cycle = g->opts.cycle > 0 ? g->opts.cycle : auto_cycle(g);
    p.gap = g->opts.gap;
    p.gr_ratio = g->opts.gr_ratio;
    p.g.layout_tag = g->layout == WBPR_BCSR ? kBCSR : kRCSR;
    p.multi_push = g->opts.multi_push;
    p.use_rev = g->layout == WBPR_BCSR ? g->opts.use_rev : 0;
    p.small_max = g->opts.small_max_degree;
    p.warp_max = g->opts.warp_max_degree;
    p.bottom_up = g->opts.bottom_up;
    p.bottom_up_min = g->opts.bottom_up_min;
    // automatic: the entry rule in phase 1 and the cut from 2^21 vertices (heights
    // beyond L2, long BFS levels over hub rows), the vertex rule below
    p.bottom_up_edges = g->opts.bottom_up_edges >= 0 ? g->opts.bottom_up_edges : (g->n >= (1LL << 21) ? 2 : 0);
    p.max_iterations = g->opts.max_iterations;
    p.timeout_ns = (unsigned long long)g->opts.barrier_timeout_ms * 1000000ull;
    if (g->opts.trace > 0) {
        if (!g->trace || g->trace_cap < g->opts.trace) {
            g->trace = (unsigned long long *)g->alloc(sizeof(unsigned long long) * 4 * (size_t)g->opts.trace, 0);
            g->trace_cap = g->trace ? g->opts.trace : 0;
        }
        p.trace = g->trace;
        p.trace_cap = g->trace_cap;
    }
    p.thread_centric = g->opts.thread_centric;
    p.barrier_extra = g->opts.barrier_extra;
    if (g->opts.warp_time) {
        if (!g->warp_ns)
            g->warp_ns = (unsigned long long *)g->alloc(sizeof(unsigned long long) * kWarps * (size_t)g->bstats_blocks, 0);
        p.warp_ns = g->warp_ns;
    }
    return p;
}

// Launch the persistent solver; stream ordered, no host synchronisation.
static wbpr_status launch_solver(wbpr_graph *g, cudaStream_t st, int mode, long long iters,
                                 unsigned char *side)
{
    const int grid = choose_grid(g);
    g->grid_blocks = grid;
    Params p = make_params(g, mode);
    p.iters_arg = iters;
    p.source_side = side;
    if (mode & kModeIters) {
        p.gap = 0;
        p.gr_ratio = 0.f;
    }
    API_CUDA(cudaMemsetAsync(g->ctl, 0, sizeof(Ctl), st));
    API_CUDA(cudaMemsetAsync(g->bstats, 0, sizeof(long long) * (size_t)grid * kStatCount, st));
    if (p.warp_ns)
        API_CUDA(cudaMemsetAsync(p.warp_ns, 0, sizeof(unsigned long long) * kWarps * (size_t)grid, st));
    API_CUDA(cudaEventRecord(g->ev0, st));
    API_CUDA(solver_launch(g->layout, g->opts.small_tile, grid, p, st, launch_smem(g)));
    API_CUDA(cudaEventRecord(g->ev1, st));
    return WBPR_OK;
}

static_assert(sizeof(Ctl) <= 64 * sizeof(long long), "the host staging buffer holds the control block");

// After a synchronised launch: read the status and counters.
static wbpr_status collect(wbpr_graph *g, cudaStream_t st, bool accumulate)
{
    long long *hp = g->pinned;
    API_CUDA(cudaMemcpyAsync(hp, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    API_CUDA(cudaStreamSynchronize(st));
    Ctl c;
    memcpy(&c, hp, sizeof(Ctl));
    std::vector<long long> bs((size_t)g->grid_blocks * kStatCount);
    API_CUDA(cudaMemcpy(bs.data(), g->bstats, sizeof(long long) * bs.size(), cudaMemcpyDeviceToHost));
    wbpr_stats s;
    memset(&s, 0, sizeof(s));
    for (int b = 0; b < g->grid_blocks; ++b) {
        const long long *x = &bs[(size_t)b * kStatCount];
        s.pushes += x[kStatPushes];
        s.relabels += x[kStatRelabels];
        s.arcs_scanned += x[kStatArcs];
        s.gr_arcs_scanned += x[kStatGrArcs];
        s.active_total += x[kStatActive];
        s.gaps += x[kStatGaps];
        s.avq_full_scans += x[kStatAvqFull];
        s.avq_bitmap_scans += x[kStatAvqInc];
        s.avq_candidates += x[kStatAvqCand];
    }
    s.iterations = c.iterations;
    s.phase1_iterations = c.phase1_iterations;
    s.global_relabels = c.global_relabels;
    s.written_off = c.written_off;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g->ev0, g->ev1);
    s.solve_ms = ms;
    if (accumulate) {
        g->stats.iterations += s.iterations;
        g->stats.global_relabels += s.global_relabels;
        g->stats.pushes += s.pushes;
        g->stats.relabels += s.relabels;
        g->stats.arcs_scanned += s.arcs_scanned;
        g->stats.gr_arcs_scanned += s.gr_arcs_scanned;
        g->stats.active_total += s.active_total;
        g->stats.gaps += s.gaps;
        g->stats.solve_ms += s.solve_ms;
    } else {
        g->stats = s;
    }
    if (c.err != 0) {
        g->solved_flow = g->solved_value = false;
        return set_error((wbpr_status)c.err, "device solve gave up (wait point " + std::to_string(c.err_where) + ")");
    }
    return WBPR_OK;
}

}  // namespace wbpr

extern "C" {

wbpr_status wbpr_maxflow(wbpr_graph *g, wbpr_stream_t stream, int64_t *value, int32_t *edge_flow)
{
    if (!g || !value) return set_error(WBPR_EINVAL, "wbpr_maxflow: NULL handle or value");
    cudaStream_t st = (cudaStream_t)stream;
    const bool want_flow = edge_flow != nullptr;
    int mode = kModePreflow | kModePhase1 | (want_flow ? kModePhase2 : 0);
    wbpr_status rc = launch_solver(g, st, mode, 0, nullptr);
    if (rc != WBPR_OK) return rc;
    rc = collect(g, st, false);
    if (rc != WBPR_OK) return rc;
    API_CUDA(cudaMemcpyAsync(g->pinned, g->e + g->t_int, sizeof(long long), cudaMemcpyDeviceToHost, st));
    if (want_flow) {
        int *mapped = is_device_ptr(edge_flow) ? nullptr : (int *)mapped_host_ptr(edge_flow);
        const bool dev = is_device_ptr(edge_flow) || mapped;
        int *out = mapped ? mapped : edge_flow;
        if (!dev) {
            if (!g->edge_tmp) {
                g->edge_tmp = (int *)g->alloc(sizeof(int) * (size_t)(g->m > 0 ? g->m : 1), st);
                if (!g->edge_tmp) return set_error(WBPR_ENOMEM, "wbpr_maxflow: staging allocation failed");
            }
            out = g->edge_tmp;
        }
        API_CUDA(launch_edge_flow(g->layout, g->m, g->arc2slot, g->cf0, g->cf, g->bf, g->prefix,
                                  g->cap_in, out, st));
        if (!dev && g->m > 0)
            API_CUDA(cudaMemcpyAsync(edge_flow, out, sizeof(int) * (size_t)g->m, cudaMemcpyDeviceToHost, st));
    }
    API_CUDA(cudaStreamSynchronize(st));
    *value = g->pinned[0];
    g->solved_value = true;
    g->solved_flow = want_flow;
    return WBPR_OK;
}

wbpr_status wbpr_maxflow_async(wbpr_graph *g, wbpr_stream_t stream, int64_t *d_value, int32_t *d_edge_flow)
{
    if (!g || !d_value) return set_error(WBPR_EINVAL, "wbpr_maxflow_async: NULL handle or value");
    cudaStream_t st = (cudaStream_t)stream;
    const bool want_flow = d_edge_flow != nullptr;
    int mode = kModePreflow | kModePhase1 | (want_flow ? kModePhase2 : 0);
    wbpr_status rc = launch_solver(g, st, mode, 0, nullptr);
    if (rc != WBPR_OK) return rc;
    API_CUDA(cudaMemcpyAsync(d_value, g->e + g->t_int, sizeof(long long), cudaMemcpyDeviceToDevice, st));
    if (want_flow)
        API_CUDA(launch_edge_flow(g->layout, g->m, g->arc2slot, g->cf0, g->cf, g->bf, g->prefix,
                                  g->cap_in, d_edge_flow, st));
    g->solved_value = true;
    g->solved_flow = want_flow;
    return WBPR_OK;
}

wbpr_status wbpr_solve_status(wbpr_graph *g, wbpr_stream_t stream)
{
    if (!g) return set_error(WBPR_EINVAL, "wbpr_solve_status: NULL handle");
    return collect(g, (cudaStream_t)stream, false);
}

wbpr_status wbpr_mincut(wbpr_graph *g, wbpr_stream_t stream, int64_t *cut_value, uint8_t *source_side)
{
    if (!g || !cut_value) return set_error(WBPR_EINVAL, "wbpr_mincut: NULL handle or cut_value");
    cudaStream_t st = (cudaStream_t)stream;
    int mode = kModeCut;
    if (!g->solved_flow) mode |= kModePreflow | kModePhase1 | kModePhase2;
    unsigned char *side = nullptr;
    unsigned char *mapped = source_side && !is_device_ptr(source_side)
                                ? (unsigned char *)mapped_host_ptr(source_side) : nullptr;
    const bool dev = source_side && (is_device_ptr(source_side) || mapped);
    if (source_side) {
        if (dev) {
            side = mapped ? mapped : source_side;
        } else {
            if (!g->side_tmp) {
                g->side_tmp = (unsigned char *)g->alloc((size_t)g->n, st);
                if (!g->side_tmp) return set_error(WBPR_ENOMEM, "wbpr_mincut: staging allocation failed");
            }
            side = g->side_tmp;
        }
    }
    wbpr_status rc = launch_solver(g, st, mode, 0, side);
    if (rc != WBPR_OK) return rc;
    rc = collect(g, st, false);
    if (rc != WBPR_OK) return rc;
    API_CUDA(cudaMemcpyAsync(g->pinned, &g->ctl->cut_value, sizeof(long long), cudaMemcpyDeviceToHost, st));
    if (source_side && !dev)
        API_CUDA(cudaMemcpyAsync(source_side, side, (size_t)g->n, cudaMemcpyDeviceToHost, st));
    API_CUDA(cudaStreamSynchronize(st));
    *cut_value = g->pinned[0];
    g->solved_flow = true;
    g->solved_value = true;
    return WBPR_OK;
}

wbpr_status wbpr_run_stage(wbpr_graph *g, wbpr_stream_t stream, int32_t stage, int64_t arg)
{
    if (!g) return set_error(WBPR_EINVAL, "wbpr_run_stage: NULL handle");
    cudaStream_t st = (cudaStream_t)stream;
    int mode;
    switch (stage) {
    case WBPR_STAGE_PREFLOW: mode = kModePreflow; break;
    case WBPR_STAGE_GLOBAL_RELABEL: mode = kModeGrOnce; break;
    case WBPR_STAGE_ITERATIONS:
        if (arg < 0) return set_error(WBPR_EINVAL, "wbpr_run_stage: negative iteration count");
        mode = kModeIters;
        break;
    default: return set_error(WBPR_EINVAL, "wbpr_run_stage: unknown stage");
    }
    // Stages continue from the current device state: the control block keeps
    // Excess_total across stage launches.
    const int grid = choose_grid(g);
    g->grid_blocks = grid;
    Params p = make_params(g, mode);
    p.iters_arg = arg;
    if (mode & kModeIters) {
        p.gap = 0;
        p.gr_ratio = 0.f;
    }
    long long keep[3] = {0, 0, 0};
    if (mode != kModePreflow) {
        Ctl c;
        API_CUDA(cudaMemcpy(&c, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
        keep[0] = c.excess_total;
        keep[1] = c.preflow_total;
        keep[2] = c.written_off;
    }
    API_CUDA(cudaMemsetAsync(g->ctl, 0, sizeof(Ctl), st));
    if (mode != kModePreflow) {
        API_CUDA(cudaMemcpyAsync(&g->ctl->excess_total, &keep[0], sizeof(long long), cudaMemcpyHostToDevice, st));
        API_CUDA(cudaMemcpyAsync(&g->ctl->preflow_total, &keep[1], sizeof(long long), cudaMemcpyHostToDevice, st));
        API_CUDA(cudaMemcpyAsync(&g->ctl->written_off, &keep[2], sizeof(long long), cudaMemcpyHostToDevice, st));
    }
    API_CUDA(cudaMemsetAsync(g->bstats, 0, sizeof(long long) * (size_t)grid * kStatCount, st));
    if (p.warp_ns)
        API_CUDA(cudaMemsetAsync(p.warp_ns, 0, sizeof(unsigned long long) * kWarps * (size_t)grid, st));
    API_CUDA(cudaEventRecord(g->ev0, st));
    API_CUDA(solver_launch(g->layout, g->opts.small_tile, grid, p, st, launch_smem(g)));
    API_CUDA(cudaEventRecord(g->ev1, st));
    g->solved_flow = g->solved_value = false;
    return collect(g, st, false);
}

wbpr_status wbpr_export(const wbpr_graph *g, int32_t what, void *host_dst, int64_t count)
{
    if (!g || (!host_dst && count > 0) || count < 0) return set_error(WBPR_EINVAL, "wbpr_export: bad arguments");
    const void *src = nullptr;
    size_t elem = 4;
    int64_t avail = 0;
    switch (what) {
    case WBPR_ARRAY_HEIGHT: src = g->h; avail = g->n; break;
    case WBPR_ARRAY_EXCESS: src = g->e; elem = 8; avail = g->n; break;
    case WBPR_ARRAY_OFFSETS: src = g->off; elem = 8; avail = g->n + 1; break;
    case WBPR_ARRAY_COL: src = g->col; avail = g->slots; break;
    case WBPR_ARRAY_CF: src = g->cf; avail = g->slots; break;
    case WBPR_ARRAY_CAP: src = g->cf0; avail = g->slots; break;
    case WBPR_ARRAY_REV: src = g->rev; avail = g->rev ? g->slots : 0; break;
    case WBPR_ARRAY_BF: src = g->bf; avail = g->bf ? g->slots : 0; break;
    case WBPR_ARRAY_IN_OFFSETS: src = g->in_off; elem = 8; avail = g->in_off ? g->n + 1 : 0; break;
    case WBPR_ARRAY_IN_COL: src = g->in_col; avail = g->in_col ? g->slots : 0; break;
    case WBPR_ARRAY_FLOW_IDX: src = g->flow_idx; avail = g->flow_idx ? g->slots : 0; break;
    case WBPR_ARRAY_ARC2SLOT: src = g->arc2slot; avail = g->m; break;
    case WBPR_ARRAY_EXCESS_TOTAL: src = &g->ctl->excess_total; elem = 8; avail = 1; break;
    case WBPR_ARRAY_TRACE_LEN: src = &g->ctl->trace_len; elem = 4; avail = 1; break;
    case WBPR_ARRAY_ORDER: src = g->order; avail = g->order ? g->n : 0; break;
    case WBPR_ARRAY_WARP_TIME: src = g->warp_ns; elem = 8; avail = g->warp_ns ? (int64_t)kWarps * g->grid_blocks : 0; break;
    case WBPR_ARRAY_ST: {
        static_assert(sizeof(int32_t) == 4, "");
        int32_t *out = (int32_t *)host_dst;
        if (count > 2) return set_error(WBPR_EINVAL, "wbpr_export: count exceeds the array");
        if (count > 0) out[0] = g->s_int;
        if (count > 1) out[1] = g->t_int;
        return WBPR_OK;
    }
    case WBPR_ARRAY_TRACE: {
        unsigned len = 0;
        if (g->trace) API_CUDA(cudaMemcpy(&len, &g->ctl->trace_len, sizeof(len), cudaMemcpyDeviceToHost));
        src = g->trace;
        elem = 8;
        avail = 4 * (int64_t)len;
        break;
    }
    default: return set_error(WBPR_EINVAL, "wbpr_export: unknown array");
    }
    if (count > avail) return set_error(WBPR_EINVAL, "wbpr_export: count exceeds the array");
    if (count == 0) return WBPR_OK;
    API_CUDA(cudaDeviceSynchronize());
    API_CUDA(cudaMemcpy(host_dst, src, elem * (size_t)count, cudaMemcpyDeviceToHost));
    return WBPR_OK;
}

}  // extern "C"
