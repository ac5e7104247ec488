// Host side of the persistent server (continuous batching).
//
// Requests and results travel through host-mapped pinned memory: the host
// writes a request's solver parameters into the ring of its size class,
// then (after a release fence) the ring's published count; a team waiting in
// the kernel sees the count with a system-scope acquire load.  Results come
// back the same way, with a `done` word written last.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "handle.h"
#include "wbpr.h"

using namespace wbpr;

struct wbpr_server {
    int device = 0;
    int layout = 0;
    cudaStream_t stream = nullptr;
    wbpr_server_options opts;
    // host-mapped
    Params *h_ring[2] = {nullptr, nullptr};
    ServerOut *h_out[2] = {nullptr, nullptr};
    unsigned *h_avail = nullptr;  // [2]
    int *h_stop = nullptr;
    // device
    unsigned char *d_ctl = nullptr;
    size_t d_ctl_bytes = 0;
    unsigned published[2] = {0, 0};
    int teams = 0;
    std::vector<wbpr_graph *> graphs[2];
    std::mutex mu;
    bool running = false;
};

namespace {

void free_server(wbpr_server *s)
{
    for (int c = 0; c < 2; ++c) {
        if (s->h_ring[c]) cudaFreeHost(s->h_ring[c]);
        if (s->h_out[c]) cudaFreeHost(s->h_out[c]);
    }
    if (s->h_avail) cudaFreeHost(s->h_avail);
    if (s->h_stop) cudaFreeHost(s->h_stop);
    if (s->d_ctl) cudaFree(s->d_ctl);
    if (s->stream) cudaStreamDestroy(s->stream);
    cudaGetLastError();
    delete s;
}

template <class T>
T *dev_ptr(T *host)
{
    void *d = nullptr;
    if (cudaHostGetDevicePointer(&d, host, 0) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (T *)d;
}

}  // namespace

extern "C" {

void wbpr_server_default_options(wbpr_server_options *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->layout = WBPR_BCSR;
    o->capacity = 1 << 16;
    o->team_blocks = 16;
    o->big_teams = 4;
    o->small_blocks = 88;    // 152 blocks = 1 per SM on a GB300: see wbpr.h
    o->idle_ms = 60000;
    o->big_slots = 1 << 15;
    o->build_room = 1;
}

}  // extern "C"

namespace {

// CUDA loads modules lazily, on a kernel's first launch, and a module load
// waits for the kernels already running -- the persistent server kernel,
// which waits for requests whose builds would need that load: a deadlock
// until the idle limit.  So before the server starts, every kernel a build
// can launch is loaded: throw-away builds of the server's layout, one tiny
// and one past the single-tile sizes of the sort and scan routines, each
// with a parallel arc (the duplicate-prefix kernels) and with both the lean
// and the default builder tuning.
wbpr_status preload_build_kernels(int layout)
{
    static std::mutex mu;
    static bool done[2] = {false, false};
    std::lock_guard<std::mutex> lock(mu);
    const int k = layout == WBPR_BCSR ? 1 : 0;
    if (done[k]) return WBPR_OK;
    for (int lean = 0; lean < 2; ++lean)
        for (int64_t m : {(int64_t)3, (int64_t)1 << 17}) {
            const int64_t n = m + 2;
            std::vector<int32_t> src((size_t)m), dst((size_t)m), cap((size_t)m, 1);
            for (int64_t i = 0; i < m; ++i) {
                src[(size_t)i] = (int32_t)(i % n);
                dst[(size_t)i] = (int32_t)((i * 7 + 1) % n);
            }
            src[(size_t)m - 1] = src[0];  // a parallel arc
            dst[(size_t)m - 1] = dst[0];
            wbpr_options o;
            wbpr_default_options(&o);
            o.lean_build = lean;
            wbpr_graph *g = wbpr_build_ex(n, m, src.data(), dst.data(), cap.data(), 0, 1, (wbpr_layout)layout, &o,
                                          nullptr);
            if (!g) return wbpr_last_error();
            int64_t v = 0;
            wbpr_status rc = wbpr_maxflow(g, nullptr, &v, nullptr);
            wbpr_destroy(g);
            if (rc != WBPR_OK) return rc;
        }
    done[k] = true;
    return WBPR_OK;
}

wbpr_server *server_start_impl(const wbpr_server_options &o)
{
    if ((o.layout != WBPR_BCSR && o.layout != WBPR_RCSR) || o.capacity < 1 || o.team_blocks < 1 ||
        o.team_blocks > 64 || (o.team_blocks & (o.team_blocks - 1)) || o.big_teams < 0 || o.small_blocks < 0 ||
        o.big_teams + o.small_blocks < 1 || o.idle_ms < 1 || o.big_slots < 0 || o.build_room < 0 ||
        o.build_room > 1) {
        set_error(WBPR_EINVAL, "wbpr_server_start: invalid options");
        return nullptr;
    }
    if (preload_build_kernels(o.layout) != WBPR_OK) return nullptr;
    wbpr_server *s = new wbpr_server();
    s->opts = o;
    s->layout = o.layout;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        set_error(WBPR_ECUDA, "wbpr_server_start: no CUDA device");
        return nullptr;
    }
    const int layout = o.layout == WBPR_BCSR ? kBCSR : kRCSR;
    int per_sm = 0, sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    if (server_max_blocks_per_sm(layout, &per_sm, o.build_room != 0) != cudaSuccess) {
        cudaGetLastError();
        free_server(s);
        set_error(WBPR_ECUDA, "wbpr_server_start: occupancy query failed");
        return nullptr;
    }
    const long long grid = (long long)o.big_teams * o.team_blocks + o.small_blocks;
    if (grid > (long long)per_sm * sms) {
        free_server(s);
        set_error(WBPR_EINVAL, "wbpr_server_start: more blocks than can be resident (" +
                                   std::to_string(per_sm * sms) + ")");
        return nullptr;
    }
    const unsigned flags = cudaHostAllocMapped | cudaHostAllocPortable;
    bool ok = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess;
    for (int c = 0; c < 2 && ok; ++c) {
        ok = cudaHostAlloc((void **)&s->h_ring[c], sizeof(Params) * (size_t)o.capacity, flags) == cudaSuccess &&
             cudaHostAlloc((void **)&s->h_out[c], sizeof(ServerOut) * (size_t)o.capacity, flags) == cudaSuccess;
        if (ok) memset(s->h_out[c], 0, sizeof(ServerOut) * (size_t)o.capacity);
    }
    ok = ok && cudaHostAlloc((void **)&s->h_avail, 2 * sizeof(unsigned), flags) == cudaSuccess &&
         cudaHostAlloc((void **)&s->h_stop, sizeof(int), flags) == cudaSuccess;
    const long long teams = (long long)o.big_teams + o.small_blocks;
    s->d_ctl_bytes = 256 + 16 * (size_t)teams;   // counters, team barriers, items, exit reasons
    ok = ok && cudaMalloc((void **)&s->d_ctl, s->d_ctl_bytes) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_server(s);
        set_error(WBPR_ENOMEM, "wbpr_server_start: allocation failed");
        return nullptr;
    }
    s->h_avail[0] = s->h_avail[1] = 0;
    *s->h_stop = 0;
    ServerDesc d;
    memset(&d, 0, sizeof(d));
    for (int c = 0; c < 2; ++c) {
        d.ring[c] = dev_ptr(s->h_ring[c]);
        d.out[c] = dev_ptr(s->h_out[c]);
        d.capacity[c] = (unsigned)o.capacity;
        d.next[c] = (unsigned *)(s->d_ctl + 4 * c);
    }
    d.mirror = (unsigned *)(s->d_ctl + 64);      // 8-byte aligned words at 64..83
    d.poll_token = (int *)(s->d_ctl + 128);
    d.avail[0] = dev_ptr(s->h_avail);
    d.avail[1] = d.avail[0] ? d.avail[0] + 1 : nullptr;
    d.stop = dev_ptr(s->h_stop);
    d.team_bar = (unsigned long long *)(s->d_ctl + 256);
    d.team_item = (unsigned *)(s->d_ctl + 256 + 8 * (size_t)teams);
    d.team_exit = (int *)(s->d_ctl + 256 + 12 * (size_t)teams);
    s->teams = (int)teams;
    d.team_big = o.team_blocks;
    d.n_big_teams = o.big_teams;
    d.idle_ns = (unsigned long long)o.idle_ms * 1000000ull;
    d.timeout_ns = 20000ull * 1000000ull;
    if (!d.ring[0] || !d.ring[1] || !d.out[0] || !d.out[1] || !d.avail[0] || !d.stop) {
        free_server(s);
        set_error(WBPR_ECUDA, "wbpr_server_start: host memory is not mapped for the device");
        return nullptr;
    }
    cudaError_t e = cudaMemsetAsync(s->d_ctl, 0, s->d_ctl_bytes, s->stream);
    if (e == cudaSuccess) e = server_launch(layout, (int)grid, d, s->stream, o.build_room != 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_server(s);
        set_error(WBPR_ECUDA, std::string("wbpr_server_start: ") + cudaGetErrorString(e));
        return nullptr;
    }
    s->running = true;
    return s;
}

int64_t server_submit_impl(wbpr_server *s, wbpr_graph *g, int mode)
{
    if (!s || !g) return set_error(WBPR_EINVAL, "wbpr_server_submit: NULL argument");
    if (g->layout != s->layout) return set_error(WBPR_ESTATE, "wbpr_server_submit: layout differs from the server's");
    std::lock_guard<std::mutex> lock(s->mu);
    if (!s->running) return set_error(WBPR_ESTATE, "wbpr_server_submit: server stopped");
    const int cls = g->slots > s->opts.big_slots && s->opts.big_teams > 0 ? 1 : 0;
    if (cls == 1 && s->opts.big_teams == 0) return set_error(WBPR_ESTATE, "wbpr_server_submit: no large teams");
    if (cls == 0 && s->opts.small_blocks == 0) return set_error(WBPR_ESTATE, "wbpr_server_submit: no small teams");
    const unsigned i = s->published[cls];
    if (i >= (unsigned)s->opts.capacity) return set_error(WBPR_ESTATE, "wbpr_server_submit: ring full");
    s->h_ring[cls][i] = make_params(g, mode);
    s->h_ring[cls][i].warp_ns = nullptr;  // the per-warp record is zeroed only by single launches
    g->grid_blocks = cls ? s->opts.team_blocks : 1;
    s->graphs[cls].push_back(g);
    std::atomic_thread_fence(std::memory_order_release);
    s->published[cls] = i + 1;
    ((volatile unsigned *)s->h_avail)[cls] = i + 1;
    return ((int64_t)cls << 40) | i;
}

// Raise the stop flag and wait for the kernel; results stay readable.
wbpr_status server_halt(wbpr_server *s)
{
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->running = false;
        std::atomic_thread_fence(std::memory_order_release);
        *(volatile int *)s->h_stop = 1;
    }
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(WBPR_ECUDA, std::string("server: ") + cudaGetErrorString(e));
    }
    return WBPR_OK;
}

}  // namespace

extern "C" {

wbpr_server *wbpr_server_start(const wbpr_server_options *opts)
{
    wbpr_server_options o;
    wbpr_server_default_options(&o);
    if (opts) o = *opts;
    return server_start_impl(o);
}

int64_t wbpr_server_submit(wbpr_server *s, wbpr_graph *g)
{
    return server_submit_impl(s, g, kModePreflow | kModePhase1);
}

wbpr_status wbpr_server_poll(wbpr_server *s, int64_t ticket, int64_t *value)
{
    if (!s || ticket < 0) return set_error(WBPR_EINVAL, "wbpr_server_poll: bad arguments");
    const int cls = (int)(ticket >> 40);
    const unsigned i = (unsigned)(ticket & ((1ll << 40) - 1));
    wbpr_graph *g = nullptr;
    {
        // A submit on another host thread may grow graphs[cls] meanwhile.
        std::lock_guard<std::mutex> lock(s->mu);
        if (cls > 1 || i >= s->published[cls]) return set_error(WBPR_EINVAL, "wbpr_server_poll: unknown ticket");
        g = s->graphs[cls][i];
    }
    volatile ServerOut *o = s->h_out[cls] + i;
    if (o->done == 0) {
        // still pending -- unless the kernel is gone (stopped, idle timeout, error)
        cudaError_t q = cudaStreamQuery(s->stream);
        if (q == cudaErrorNotReady) return (wbpr_status)1;
        cudaGetLastError();
        if (o->done == 0)
            return set_error(WBPR_ESTATE, std::string("wbpr_server_poll: the server kernel has exited (") +
                                              cudaGetErrorString(q) + "; a team gives up after idle_ms without requests)");
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    memset(&g->stats, 0, sizeof(g->stats));
    g->stats.iterations = o->iterations;
    g->stats.solve_ms = (double)(o->t_end - o->t_start) * 1e-6;
    if (o->err != 0) return set_error((wbpr_status)o->err, "wbpr_server_poll: device solve gave up");
    if (value) *value = o->value;
    g->solved_value = true;
    g->solved_flow = false;
    return WBPR_OK;
}

wbpr_status wbpr_server_times(wbpr_server *s, int64_t ticket, uint64_t *t_start_ns, uint64_t *t_end_ns)
{
    if (!s || ticket < 0 || !t_start_ns || !t_end_ns) return set_error(WBPR_EINVAL, "wbpr_server_times: bad arguments");
    const int cls = (int)(ticket >> 40);
    const unsigned i = (unsigned)(ticket & ((1ll << 40) - 1));
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (cls > 1 || i >= s->published[cls]) return set_error(WBPR_EINVAL, "wbpr_server_times: unknown ticket");
    }
    volatile ServerOut *o = s->h_out[cls] + i;
    if (o->done == 0) return (wbpr_status)1;
    std::atomic_thread_fence(std::memory_order_acquire);
    *t_start_ns = o->t_start;
    *t_end_ns = o->t_end;
    return WBPR_OK;
}

wbpr_status wbpr_server_team_exits(wbpr_server *s, int32_t *reasons, int32_t count)
{
    if (!s || count < 0 || count > s->teams || (count && !reasons))
        return set_error(WBPR_EINVAL, "wbpr_server_team_exits: bad arguments");
    if (cudaStreamQuery(s->stream) == cudaErrorNotReady) return (wbpr_status)1;
    cudaGetLastError();
    if (count && cudaMemcpy(reasons, s->d_ctl + 256 + 12 * (size_t)s->teams, sizeof(int32_t) * (size_t)count,
                            cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return set_error(WBPR_ECUDA, "wbpr_server_team_exits: copy failed");
    }
    return WBPR_OK;
}

wbpr_status wbpr_server_stop(wbpr_server *s)
{
    if (!s) return WBPR_OK;
    wbpr_status rc = server_halt(s);
    free_server(s);
    return rc;
}

// Batched solves through the server: every handle is published at once
// (largest first within its size class); large instances go to teams of
// batch_team blocks, small ones to single-block teams, and the two classes
// share the grid in proportion to their residual slots.
wbpr_status wbpr_maxflow_batch(wbpr_graph *const *gs, int32_t count, wbpr_stream_t stream, int64_t *values,
                               int32_t *const *edge_flows)
{
    if (count < 0 || (count > 0 && (!gs || !values)))
        return set_error(WBPR_EINVAL, "wbpr_maxflow_batch: bad arguments");
    int device = 0;
    if (count > 0 && cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return set_error(WBPR_ECUDA, "wbpr_maxflow_batch: no CUDA device");
    }
    for (int i = 0; i < count; ++i) {
        if (!gs[i]) return set_error(WBPR_ESTATE, "wbpr_maxflow_batch: NULL handle");
        if (gs[i]->device != device) return set_error(WBPR_ESTATE, "wbpr_maxflow_batch: handle of another device");
    }
    {
        std::vector<const wbpr_graph *> sorted(gs, gs + count);
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
            return set_error(WBPR_ESTATE, "wbpr_maxflow_batch: repeated handle");
    }
    if (count == 0) return WBPR_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return set_error(WBPR_ECUDA, "wbpr_maxflow_batch: stream error");
    }
    const wbpr_options &bo = gs[0]->opts;
    wbpr_status rc = WBPR_OK;
    for (int lay = 0; lay < 2; ++lay) {
        std::vector<int> big, small;
        double w_big = 0, w_all = 0;
        for (int i = 0; i < count; ++i) {
            if ((gs[i]->layout == WBPR_BCSR) != (lay == 1)) continue;
            const double w = (double)gs[i]->slots + (double)gs[i]->n;
            w_all += w;
            if (gs[i]->slots > bo.batch_big_slots) {
                big.push_back(i);
                w_big += w;
            } else {
                small.push_back(i);
            }
        }
        if (big.empty() && small.empty()) continue;
        auto by_size = [&](int a, int b) { return gs[a]->slots > gs[b]->slots; };
        std::stable_sort(big.begin(), big.end(), by_size);
        std::stable_sort(small.begin(), small.end(), by_size);
        const int layout = lay ? kBCSR : kRCSR;
        int per_sm = 0;
        if (server_max_blocks_per_sm(layout, &per_sm, false) != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            return set_error(WBPR_ECUDA, "wbpr_maxflow_batch: occupancy query failed");
        }
        long long total = (long long)per_sm * gs[0]->num_sms;
        if (bo.grid_blocks > 0 && bo.grid_blocks < total) total = bo.grid_blocks;
        const int team = bo.batch_team;
        long long big_teams = 0, small_blocks = 0;
        if (!big.empty()) {
            big_teams = small.empty() ? total / team : (long long)(w_big / w_all * (double)total / team + 0.5);
            if (big_teams < 1) big_teams = 1;
            if (big_teams > (long long)big.size()) big_teams = (long long)big.size();
            if (big_teams * team > total) big_teams = total / team;
        }
        if (!small.empty()) {
            small_blocks = total - big_teams * team;
            if (small_blocks < 1) {
                big_teams = big_teams > 1 ? big_teams - 1 : 0;
                small_blocks = total - big_teams * team;
            }
            if (small_blocks > (long long)small.size()) small_blocks = (long long)small.size();
        }
        if (big_teams == 0 && !big.empty()) {
            // no room for a team: solve the large ones on single blocks too
            small.insert(small.begin(), big.begin(), big.end());
            big.clear();
            small_blocks = total < (long long)small.size() ? total : (long long)small.size();
        }
        wbpr_server_options o;
        wbpr_server_default_options(&o);
        o.layout = lay ? WBPR_BCSR : WBPR_RCSR;
        o.capacity = (int32_t)(big.size() > small.size() ? big.size() : small.size());
        o.team_blocks = team;
        o.big_teams = (int32_t)big_teams;
        o.small_blocks = (int32_t)small_blocks;
        o.big_slots = bo.batch_big_slots;
        o.idle_ms = bo.barrier_timeout_ms;
        o.build_room = 0;  // nothing is built while the batch's server runs
        wbpr_server *srv = server_start_impl(o);
        if (!srv) return wbpr_last_error();
        std::vector<std::pair<int, int64_t>> tickets;
        for (const std::vector<int> *grp : {&big, &small}) {
            for (int i : *grp) {
                const bool want_flow = edge_flows && edge_flows[i];
                const int mode = kModePreflow | kModePhase1 | (want_flow ? kModePhase2 : 0);
                // route explicitly: the class follows the group, not only the size
                const int64_t saved = srv->opts.big_slots;
                srv->opts.big_slots = grp == &big ? -1 : INT64_MAX;
                const int64_t t = server_submit_impl(srv, gs[i], mode);
                srv->opts.big_slots = saved;
                if (t < 0) {
                    server_halt(srv);
                    free_server(srv);
                    return (wbpr_status)t;
                }
                tickets.push_back({i, t});
            }
        }
        wbpr_status hrc = server_halt(srv);
        for (auto &it : tickets) {
            int64_t v = 0;
            wbpr_status prc = wbpr_server_poll(srv, it.second, &v);
            if (prc == WBPR_OK) {
                values[it.first] = v;
                gs[it.first]->solved_flow = edge_flows && edge_flows[it.first];
            } else if (rc == WBPR_OK) {
                rc = prc == (wbpr_status)1 ? set_error(WBPR_ETIMEOUT, "wbpr_maxflow_batch: instance not finished")
                                           : prc;
            }
        }
        free_server(srv);
        if (hrc != WBPR_OK) return hrc;
    }
    if (rc != WBPR_OK) return rc;
    for (int i = 0; i < count; ++i) {
        if (!(edge_flows && edge_flows[i])) continue;
        wbpr_graph *g = gs[i];
        cudaError_t e = launch_edge_flow(g->layout, g->m, g->arc2slot, g->cf0, g->cf, g->bf, g->prefix, g->cap_in,
                                         edge_flows[i], st);
        if (e != cudaSuccess) return set_error(WBPR_ECUDA, std::string("wbpr_maxflow_batch: ") + cudaGetErrorString(e));
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return set_error(WBPR_ECUDA, "wbpr_maxflow_batch: stream error");
    }
    return WBPR_OK;
}

}  // extern "C"
