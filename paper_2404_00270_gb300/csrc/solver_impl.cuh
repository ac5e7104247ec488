// Persistent push-relabel solver for sm_103a.
//
// One cooperative launch runs a whole solve: reset + preflow (Alg. 1 step 0),
// the global relabel of §2.2 as a level-synchronous backward BFS from the
// sink, and the push-relabel iterations of Alg. 2 until the termination test
// of Alg. 1 (e(s) + e(t) >= Excess_total) holds on the device; optionally a
// second phase that returns stranded excess to s, and a forward BFS for the
// minimum cut.  Grid-wide synchronisation (the grid_sync() of Alg. 2) is a
// counter barrier with a time limit: a wait that gives up records
// WBPR_ETIMEOUT in the control block and every block leaves the kernel.
//
// One iteration of Alg. 2:
//   1. AVQ compaction: every block scans a contiguous range of vertices and
//      appends the active ones (e > 0, h below the height cap, not s or t) to
//      the global queue of their tile class: warp ballots rank them, a block
//      prefix over the warps places them, and one atomic per class per 1024
//      vertices reserves the block's range (the atomic_add of Alg. 2,
//      aggregated).
//   2. grid_sync.
//   3. Two-level parallelism: each active vertex is owned by one tile whose
//      width follows its residual-list length: `SW` lanes (small rows), a
//      warp, or, for hub rows, several warps that take 256-entry chunks of the
//      row dynamically.  The tile
//      scans the list coalesced, gathers neighbour heights of residual arcs,
//      and reduces (height, slot) keys to the minimum with warp shuffles;
//      the tile's lane 0 then pushes min(e(u), cf(u,v')) with atomics when
//      h(u) > h(v'), else relabels h(u) = h(v') + 1 (Alg. 1, relaxed push
//      condition of §2.2).
//   4. grid_sync.
// Only the owner of u ever lowers e(u) or a residual capacity out of u, so
// the pushed amount is always positive and no value goes negative; stale
// neighbour heights are tolerated as in the lock-free algorithm.
//
// Gap heuristic: a relabel moves u from height hu to hn and keeps per-height
// counts of vertices below n (count[], rebuilt at every global relabel from
// the BFS level sizes).  When count[hu] drops to zero the level is a gap
// candidate; at the next AVQ compaction (a quiescent point) it is re-checked
// and, if still empty, every vertex with hu < h < n is lifted to n.
// This header holds the device code; each kernel variant (layout x small
// tile width, and the server kernel per layout) is instantiated in a
// translation unit of its own (inst_*.cu) so that they compile in parallel.
#pragma once
#include <stdint.h>

#include "wbpr_internal.cuh"


namespace wbpr {
namespace {

typedef unsigned long long u64;
constexpr u64 kNoKey = ~0ULL;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ u64 ld_acquire(const u64 *p)
{
    u64 v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ u64 global_ns()
{
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_err(const Ctl *c)
{
    return *(volatile const int *)&c->err;
}

__device__ __forceinline__ u64 make_key(int h, unsigned idx)
{
    return ((u64)(unsigned)h << 32) | idx;
}

__device__ __forceinline__ u64 umin64(u64 a, u64 b) { return a < b ? a : b; }

template <int W>
__device__ __forceinline__ u64 tile_min(u64 x)
{
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) x = umin64(x, __shfl_xor_sync(kFull, x, o));
    return x;
}

constexpr int kBuVerts = 4;  // vertices per thread per bottom-up pass

struct Smem {
    int qbuf[kClasses][kQueueCap];
    int dfr[kBlock * kBuVerts];  // bottom-up BFS: rows deferred to a warp (front) or the block (back)
    unsigned ndfr_lo, ndfr_hi;
    unsigned qcnt[kClasses];
    unsigned qbase[kClasses];
    unsigned wcnt[2][kWarps];    // AVQ compaction: per-warp counts of classes 0 and 1
    unsigned gbase[2];           //                 the block's base in the global queues
    u64 red[kWarps];
    long long red64[kWarps];
    long long wsum[kWarps];
    long long bcast64;
    int bcast32;
    long long stats[kStatCount];
    int ok;
};

// Per-block view of one solve.  A solve runs on a team of `nblk` blocks:
// the whole grid for a single instance, or a slice of it in a batch; `bid`
// is this block's rank in the team.
struct Ctx {
    const Params &P;
    Smem &sm;
    u64 bar_target;  // meaningful in thread 0 only
    int gen;         // queue generation (uniform across the team)
    unsigned nblk;
    unsigned bid;
    u64 gr_start_ns, gr_ns, gr_end_ns;  // last global relabel (rank 0, thread 0)
    int *stage;      // dynamic shared memory for staging hub chunks (kStageBytes), or null
    long long fe;    // this thread's share of the next frontier's residual-list entries
};

// Asynchronous 16-byte copies global -> shared (cp.async, L2 only), and the
// waits for them: hardware waits on the thread's own copy groups.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ unsigned dynamic_smem_bytes()
{
    unsigned v;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
    return v;
}

// Grid-wide barrier with a time limit.  Returns false on any device error.
__device__ bool grid_sync(Ctx &c, int where)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        Ctl *ctl = c.P.st.ctl;
        c.bar_target += c.nblk + (unsigned)c.P.barrier_extra;
        __threadfence();
        if (c.nblk > 1) atomicAdd(&ctl->bar, 1ULL);
        int ok = 1;
        u64 t0 = 0;
        unsigned spins = 0;
        while (c.nblk > 1 && ld_acquire(&ctl->bar) < c.bar_target) {
            if (ld_err(ctl) != 0) { ok = 0; break; }
            ++spins;
            if ((spins & 255u) == 0) {
                u64 now = global_ns();
                if (t0 == 0) {
                    t0 = now;
                } else if (now - t0 > c.P.timeout_ns) {
                    atomicCAS(&ctl->err, 0, (int)WBPR_ETIMEOUT);
                    ctl->err_where = where;
                    ok = 0;
                    break;
                }
            }
            if (spins > 64) __nanosleep(20);
        }
        __threadfence();
        if (ld_err(ctl) != 0) ok = 0;
        c.sm.ok = ok;
        if (c.P.trace && c.bid == 0) {
            unsigned i = ctl->trace_len;
            if (i < (unsigned)c.P.trace_cap) {
                const unsigned *q = ctl->q_count[c.gen % 3];
                const u64 hubs = ctl->hub_pack[c.gen % 3] >> 40;
                u64 *r = c.P.trace + 4ull * i;
                r[0] = (u64)where;
                r[1] = (u64)c.gen;
                r[2] = global_ns();
                r[3] = (u64)q[0] | ((u64)q[1] << 24) | (hubs << 48);
                ctl->trace_len = i + 1;
            }
        }
    }
    __syncthreads();
    return c.sm.ok != 0;
}

template <int L>
__device__ __forceinline__ long long degree(const GraphDev &g, int v)
{
    long long d = __ldg(g.off + v + 1) - __ldg(g.off + v);
    if (L == kRCSR) d += __ldg(g.in_off + v + 1) - __ldg(g.in_off + v);
    return d;
}

// Slots between the 16-byte boundary below a BCSR row and the row's start.
template <int L>
__device__ __forceinline__ int hub_lead(const GraphDev &g, int v)
{
    return L == kBCSR ? (int)(__ldg(g.off + v) & 3) : 0;
}

__device__ __forceinline__ int classify(const Params &P, long long d)
{
    return d <= P.small_max ? 0 : (d <= P.warp_max ? 1 : 2);
}

// ---------------------------------------------------------------------------
// Queue production: stage in shared memory, flush with one atomic per class.
// ---------------------------------------------------------------------------
// The lanes of a warp that append at the same time and to the same class
// share one atomic (opportunistic aggregation: whatever lanes are converged
// here); once the block's staging is full, the overflow goes to the global
// queue, again with one atomic per group of lanes.
__device__ __forceinline__ void q_append(Ctx &c, int slot3, int set, int cls, int v)
{
    const unsigned am = __activemask();
    const unsigned same = __match_any_sync(am, cls);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(same) - 1;
    const unsigned lt = (1u << lane) - 1u;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(&c.sm.qcnt[cls], (unsigned)__popc(same));
    const unsigned pos = __shfl_sync(same, base, leader) + __popc(same & lt);
    const unsigned ov = __ballot_sync(same, pos >= (unsigned)kQueueCap);
    if (pos < (unsigned)kQueueCap) {
        c.sm.qbuf[cls][pos] = v;
    } else {
        const int l2 = __ffs(ov) - 1;
        unsigned gbase = 0;
        if (lane == l2) gbase = atomicAdd(&c.P.st.ctl->q_count[slot3][cls], (unsigned)__popc(ov));
        gbase = __shfl_sync(ov, gbase, l2);
        c.P.st.q[set][cls][gbase + __popc(ov & lt)] = v;
    }
}

// All threads of the block call this.
__device__ void q_flush(Ctx &c, int slot3, int set)
{
    __syncthreads();
    if (threadIdx.x < kClasses) {
        unsigned k = c.sm.qcnt[threadIdx.x];
        if (k > (unsigned)kQueueCap) k = kQueueCap;
        c.sm.qbase[threadIdx.x] = k ? atomicAdd(&c.P.st.ctl->q_count[slot3][threadIdx.x], k) : 0u;
        c.sm.qcnt[threadIdx.x] = k;
    }
    __syncthreads();
#pragma unroll
    for (int cls = 0; cls < kClasses; ++cls) {
        unsigned k = c.sm.qcnt[cls];
        int *dst = c.P.st.q[set][cls] + c.sm.qbase[cls];
        for (unsigned i = threadIdx.x; i < k; i += kBlock) dst[i] = c.sm.qbuf[cls][i];
    }
    __syncthreads();
    if (threadIdx.x < kClasses) c.sm.qcnt[threadIdx.x] = 0;
    __syncthreads();
}

__device__ __forceinline__ void reset_rotating(Ctx &c, int gen)
{
    if (c.bid == 0 && threadIdx.x == 0) {
        Ctl *ctl = c.P.st.ctl;
        int z = (gen + 2) % 3;
        for (int k = 0; k < kClasses; ++k) ctl->q_count[z][k] = 0;
        ctl->q_grab[z] = 0;
        ctl->q_grab_w[z] = 0;
        ctl->fedges[z] = 0;
        ctl->hub_pack[z] = 0;
        ctl->gap_level[z] = kUnvisited;
    }
}

// The counters of a block-local pass of generation gen live in slot gen % 3;
// every push-relabel pass of generation gen clears slot (gen + 1) % 3 for
// the next one (its last readers passed the barrier before this pass).
__device__ __forceinline__ void reset_local_slot(Ctx &c, int gen)
{
    if (c.bid == 0 && threadIdx.x == 0) {
        c.P.st.ctl->local_active[(gen + 1) % 3] = 0;
        c.P.st.ctl->local_defer[(gen + 1) % 3] = 0;
    }
}

// ---------------------------------------------------------------------------
// Hub class: a vertex whose residual list is longer than warp_max is split
// into chunks of kWChunk entries (push-relabel passes, BFS levels and the
// cut), each taken by one warp.  One 64-bit atomic gives it both its queue
// position and the id of its first chunk; the appender then records the
// position under each of its chunk ids, so a warp that takes a chunk id
// finds its hub with one load.  A hub's chunks start `lead` = off[u] mod 4
// slots before its row (BCSR), so that chunk boundaries fall on 16-byte
// boundaries of the slot arrays.
// ---------------------------------------------------------------------------
constexpr u64 kChunkMask = (1ull << 40) - 1;

__device__ __forceinline__ unsigned hub_chunks(long long deg, int chunk = kWChunk, int lead = 0)
{
    return deg <= 0 ? 1u : (unsigned)((deg + lead + chunk - 1) / chunk);
}

// Appends hub v; returns its queue position, and its first chunk id and
// chunk count in *first / *nch.  With fill = false the caller writes the
// chunk table (warp_fill_chunks).
__device__ __forceinline__ unsigned hub_append(Ctx &c, int slot3, int set, int v, long long deg, bool pr,
                                               long long ev, int chunk = kWChunk, int lead = 0,
                                               bool fill = true, unsigned *first_out = nullptr,
                                               unsigned *nch_out = nullptr)
{
    const StateDev &st = c.P.st;
    const unsigned nch = hub_chunks(deg, chunk, lead);
    const u64 old = atomicAdd(&st.ctl->hub_pack[slot3], (1ull << 40) | nch);
    const unsigned pos = (unsigned)(old >> 40);
    const unsigned first = (unsigned)(old & kChunkMask);
    st.q[set][2][pos] = v;
    st.hub_start[set][pos] = first;
    if (fill)
        for (unsigned j = 0; j < nch; ++j) st.hub_chunk[set][first + j] = pos;
    if (first_out) *first_out = first;
    if (nch_out) *nch_out = nch;
    if (pr) {
        st.hub_e0[set][pos] = ev;
        st.hub_rem[set][pos] = ev;
        st.hub_aux[set][pos] = kNoKey;
        st.hub_done[set][pos] = 0;
    }
    return pos;
}

// The whole warp writes the chunk table of the hubs its lanes appended (lane
// mask `hubs`): chunk id -> queue position, 32 entries per step.
__device__ __forceinline__ void warp_fill_chunks(const StateDev &st, int set, unsigned hubs, unsigned pos,
                                                 unsigned first, unsigned nch)
{
    const int lane = threadIdx.x & 31;
    while (hubs) {
        const int src = __ffs(hubs) - 1;
        hubs &= hubs - 1;
        const unsigned p = __shfl_sync(kFull, pos, src);
        const unsigned f = __shfl_sync(kFull, first, src);
        const unsigned k = __shfl_sync(kFull, nch, src);
        for (unsigned j = lane; j < k; j += 32) st.hub_chunk[set][f + j] = p;
    }
}

// Hub appends of a whole warp (all lanes call, `is_hub` on the lanes that
// append): one atomic on the hub counter for all of the warp's hubs, their
// queue positions by rank and their first chunk ids by a warp scan of their
// chunk counts (kWChunk entries, BCSR rows aligned down to 16 bytes), then
// the warp writes their chunk tables together.
template <int L>
__device__ __forceinline__ void warp_hub_append(Ctx &c, int slot3, int set, bool is_hub, int v, long long deg,
                                                long long ev)
{
    const unsigned hm = __ballot_sync(kFull, is_hub);
    if (!hm) return;
    const StateDev &st = c.P.st;
    const int lane = threadIdx.x & 31;
    const unsigned nch = is_hub ? hub_chunks(deg, kWChunk, hub_lead<L>(c.P.g, v)) : 0u;
    unsigned incl = nch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const unsigned tot = __shfl_sync(kFull, incl, 31);
    u64 base = 0;
    if (lane == 0) base = atomicAdd(&st.ctl->hub_pack[slot3], ((u64)__popc(hm) << 40) | tot);
    base = __shfl_sync(kFull, base, 0);
    const unsigned pos = (unsigned)(base >> 40) + __popc(hm & ((1u << lane) - 1u));
    const unsigned first = (unsigned)(base & kChunkMask) + incl - nch;
    if (is_hub) {
        st.q[set][2][pos] = v;
        st.hub_start[set][pos] = first;
        st.hub_e0[set][pos] = ev;
        st.hub_rem[set][pos] = ev;
        st.hub_aux[set][pos] = kNoKey;
        st.hub_done[set][pos] = 0;
    }
    warp_fill_chunks(st, set, hm, pos, first, nch);
}


__device__ __forceinline__ unsigned queue_total(const Ctl *ctl, int gen)
{
    const int s3 = gen % 3;
    return __ldcg(&ctl->q_count[s3][0]) + __ldcg(&ctl->q_count[s3][1]) +
           (unsigned)(__ldcg(&ctl->hub_pack[s3]) >> 40);
}

// Row index r of u's residual list -> slot (RCSR: out entries, then in entries).
template <int L>
__device__ __forceinline__ long long row_slot(long long ob, long long dout, long long ib, long long r,
                                              bool &in)
{
    if (L == kBCSR || r < dout) {
        in = false;
        return ob + r;
    }
    in = true;
    return ib + (r - dout);
}

__device__ long long block_sum(Ctx &c, long long x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) c.sm.red64[threadIdx.x >> 5] = x;
    __syncthreads();
    long long s = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kWarps; ++w) s += c.sm.red64[w];
    return s;  // valid in thread 0
}

// ---------------------------------------------------------------------------
// Residual-list scans.  `rounds_*` are uniform over the tile (or warp).
// BCSR: entries [b, e) of u's merged row; key index = k - b.
// RCSR: out entries first (index j - ob), then in entries (dout + k - ib).
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ u64 scan_bcsr(const GraphDev &g, const int *h, long long b,
                                         long long e, int lane, int rounds)
{
    u64 best = kNoKey;
#pragma unroll 4
    for (int r = 0; r < rounds; ++r) {
        long long k = b + (long long)r * W + lane;
        if (k < e) {
            int cfk = __ldcg(g.cf + k);
            int v = __ldg(g.col + k);
            if (cfk > 0) best = umin64(best, make_key(__ldcg(h + v), (unsigned)(k - b)));
        }
    }
    return best;
}

template <int W>
__device__ __forceinline__ u64 scan_rcsr(const GraphDev &g, const int *h, long long ob,
                                         long long oe, long long ib, long long ie, int lane,
                                         int rounds_out, int rounds_in)
{
    u64 best = kNoKey;
#pragma unroll 4
    for (int r = 0; r < rounds_out; ++r) {
        long long j = ob + (long long)r * W + lane;
        if (j < oe) {
            int c = __ldcg(g.cf + j);
            int v = __ldg(g.col + j);
            if (c > 0) best = umin64(best, make_key(__ldcg(h + v), (unsigned)(j - ob)));
        }
    }
    const unsigned dout = (unsigned)(oe - ob);
#pragma unroll 4
    for (int r = 0; r < rounds_in; ++r) {
        long long k = ib + (long long)r * W + lane;
        if (k < ie) {
            unsigned j = __ldg(g.flow_idx + k);
            int v = __ldg(g.in_col + k);
            int c = __ldcg(g.bf + j);
            if (c > 0) best = umin64(best, make_key(__ldcg(h + v), dout + (unsigned)(k - ib)));
        }
    }
    return best;
}

__device__ __forceinline__ long long lower_bound_col(const int *col, long long b, long long e,
                                                     int key)
{
    while (b < e) {
        long long mid = (b + e) >> 1;
        if (__ldg(col + mid) < key) b = mid + 1;
        else e = mid;
    }
    return b;
}

// Marks v as a candidate of the next AVQ (incremental compaction): a
// fire-and-forget atomic OR on v's bitmap word.  Pushes mark their target,
// and an owner that keeps excess after its pass marks itself, so every
// vertex that can be active after a pass is marked.
__device__ __forceinline__ void touch_mark(const StateDev &st, int v)
{
    if (st.touch) atomicOr(st.touch + (v >> 5), 1u << (v & 31));
}

// Relabel u from hu to hn (capped at hcap) and keep the gap counts.
__device__ __forceinline__ void relabel_to(Ctx &c, int u, int hu, int hn, bool phase1, int hcap)
{
    const Params &P = c.P;
    if (hn > hcap) hn = hcap;
    __stcg(P.st.h + u, hn);
    atomicAdd((unsigned long long *)&c.sm.stats[kStatRelabels], 1ull);
    if (phase1 && P.gap) {
        int *count = P.st.count;
        const int n = P.g.n;
        if (hn < n) atomicAdd(count + hn, 1);
        int prev = atomicSub(count + hu, 1);
        if (prev == 1) atomicMin(&P.st.ctl->gap_level[c.gen % 3], hu);
    }
}

// Push or relabel for the owner of u (one thread).  Alg. 1: if h(u) > h'
// push d = min(e(u), cf(u, v')) with four atomics, else h(u) = h' + 1.
template <int L>
__device__ void apply_op(Ctx &c, int u, u64 key, bool phase1, int hcap)
{
    const Params &P = c.P;
    const GraphDev &g = P.g;
    int *h = P.st.h;
    long long *e = P.st.e;
    const int hu = __ldcg(h + u);
    if (key != kNoKey) {
        const int hmin = (int)(key >> 32);
        const unsigned idx = (unsigned)(key & 0xffffffffu);
        if (hu > hmin) {
            long long eu = __ldcg(e + u);
            int v;
            int *dec;
            int *inc;
            long long mir_a = -1, mir_ra = -1;
            if (L == kBCSR) {
                long long a = __ldg(g.off + u) + idx;
                v = __ldg(g.col + a);
                long long ra;
                if (P.use_rev) {
                    ra = __ldg(g.rev + a);
                } else {
                    ra = lower_bound_col(g.col, __ldg(g.off + v), __ldg(g.off + v + 1), u);
                }
                dec = g.cf + a;
                inc = g.cf + ra;
                mir_a = a;
                mir_ra = ra;
            } else {
                long long ob = __ldg(g.off + u);
                unsigned dout = (unsigned)(__ldg(g.off + u + 1) - ob);
                if (idx < dout) {
                    long long j = ob + idx;
                    v = __ldg(g.col + j);
                    dec = g.cf + j;
                    inc = g.bf + j;
                } else {
                    long long k = __ldg(g.in_off + u) + (idx - dout);
                    unsigned j = __ldg(g.flow_idx + k);
                    v = __ldg(g.in_col + k);
                    dec = g.bf + j;
                    inc = g.cf + j;
                }
            }
            int cav = __ldcg(dec);
            long long d = eu < (long long)cav ? eu : (long long)cav;
            if (d > 0) {
                atomicSub(dec, (int)d);
                atomicAdd((u64 *)(e + u), (u64)(-d));
                atomicAdd(inc, (int)d);
                if (L == kBCSR && g.cfb) {
                    atomicAdd(g.cfb + mir_a, (int)d);
                    atomicSub(g.cfb + mir_ra, (int)d);
                }
                atomicAdd((u64 *)(e + v), (u64)d);
                touch_mark(P.st, v);
                atomicAdd((unsigned long long *)&c.sm.stats[kStatPushes], 1ull);
            }
            if (eu > d) touch_mark(P.st, u);
            return;
        }
    }
    int hn = (key == kNoKey) ? hcap : (int)(key >> 32) + 1;
    relabel_to(c, u, hu, hn, phase1, hcap);
    touch_mark(P.st, u);
}

// Tile of W <= 32 lanes (all 32 lanes of the warp call this; u < 0 = idle).
template <int L, int W>
__device__ void pr_tile(Ctx &c, int u, int sl, bool phase1, int hcap)
{
    const GraphDev &g = c.P.g;
    long long ob = 0, oe = 0, ib = 0, ie = 0;
    int ro = 0, ri = 0;
    if (u >= 0) {
        ob = __ldg(g.off + u);
        oe = __ldg(g.off + u + 1);
        ro = (int)((oe - ob + W - 1) / W);
        if (L == kRCSR) {
            ib = __ldg(g.in_off + u);
            ie = __ldg(g.in_off + u + 1);
            ri = (int)((ie - ib + W - 1) / W);
        }
    }
    ro = __reduce_max_sync(kFull, ro);
    if (L == kRCSR) ri = __reduce_max_sync(kFull, ri);
    u64 best = (L == kBCSR) ? scan_bcsr<W>(g, c.P.st.h, ob, oe, sl, ro)
                            : scan_rcsr<W>(g, c.P.st.h, ob, oe, ib, ie, sl, ro, ri);
    best = tile_min<W>(best);
    if (u >= 0 && sl == 0) {
        atomicAdd((unsigned long long *)&c.sm.stats[kStatArcs], (u64)((oe - ob) + (ie - ib)));
        apply_op<L>(c, u, best, phase1, hcap);
    }
}

// ---------------------------------------------------------------------------
// Discharge pass (multi-push).  The owner tile of u reads e(u) = E and h(u)
// once, then walks u's residual list: every arc read as lower (cf > 0 and
// h(v) < h(u)) is admissible, and the tile splits the remaining excess over
// the admissible arcs of each chunk in slot order with an inclusive prefix
// sum of their capacities, so every lane pushes min(cf, what is left before
// it).  Each push is the push of Alg. 1 (relaxed condition h(u) > h(v) on
// the heights read); several of them per pass replace one push per
// iteration.  If excess is left after the whole list, every arc still
// residual was read at a height >= h(u) and u is relabelled to one above the
// lowest of them.  The pass stops reading as soon as the excess is gone.
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ long long seg_incl_scan(long long x, int sl)
{
#pragma unroll
    for (int o = 1; o < W; o <<= 1) {
        long long y = __shfl_up_sync(kFull, x, o, W);
        if (sl >= o) x += y;
    }
    return x;
}

template <int W>
__device__ __forceinline__ int seg_min_int(int x)
{
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) {
        int y = __shfl_xor_sync(kFull, x, o);
        x = y < x ? y : x;
    }
    return x;
}

template <int W>
__device__ __forceinline__ int seg_sum_int(int x)
{
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// Load entry k of u's list: residual capacity and neighbour (and its height
// when residual).  `in` selects the RCSR in-list.
template <int L>
__device__ __forceinline__ void mp_load(const Params &P, long long k, bool in, int &cap, int &v,
                                        int &hv)
{
    const GraphDev &g = P.g;
    if (L == kRCSR && in) {
        unsigned j = __ldg(g.flow_idx + k);
        cap = __ldcg(g.bf + j);
        v = __ldg(g.in_col + k);
    } else {
        cap = __ldcg(g.cf + k);
        v = __ldg(g.col + k);
    }
    hv = cap > 0 ? __ldcg(P.st.h + v) : 0x7fffffff;
}

// Push d along entry k of u's list.
template <int L>
__device__ __forceinline__ void mp_push(const Params &P, int u, long long k, bool in, int v, int d)
{
    const GraphDev &g = P.g;
    int *dec;
    int *inc;
    if (L == kBCSR) {
        long long ra = P.use_rev ? (long long)__ldg(g.rev + k)
                                 : lower_bound_col(g.col, __ldg(g.off + v), __ldg(g.off + v + 1), u);
        dec = g.cf + k;
        inc = g.cf + ra;
        if (g.cfb) {
            atomicAdd(g.cfb + k, d);
            atomicSub(g.cfb + ra, d);
        }
    } else if (!in) {
        dec = g.cf + k;
        inc = g.bf + k;
    } else {
        unsigned j = __ldg(g.flow_idx + k);
        dec = g.bf + j;
        inc = g.cf + j;
    }
    atomicSub(dec, d);
    atomicAdd(inc, d);
    atomicAdd((u64 *)(P.st.e + v), (u64)(long long)d);
    touch_mark(P.st, v);
}

template <int L, int W>
__device__ __forceinline__ void mp_list(Ctx &c, int u, long long b, long long e, int rounds, bool in,
                                        int sl, int hu, long long &rem, int &hres, int &npush,
                                        long long &scanned)
{
    // Groups of kIlp rounds: all loads of a group are issued before the
    // (sequential) prefix-sum steps, so kIlp memory chains are in flight.
    constexpr int kIlp = 4;
    const Params &P = c.P;
    const GraphDev &g = P.g;
    for (int r0 = 0; r0 < rounds; r0 += kIlp) {
        if (__all_sync(kFull, rem == 0)) break;
        int cap[kIlp], v[kIlp], hv[kIlp];
#pragma unroll
        for (int q = 0; q < kIlp; ++q) {
            const long long base = b + (long long)(r0 + q) * W;
            const long long k = base + sl;
            cap[q] = 0;
            v[q] = 0;
            hv[q] = 0x7fffffff;
            if (rem > 0 && r0 + q < rounds && k < e) {
                if (L == kRCSR && in) {
                    const unsigned j = __ldg(g.flow_idx + k);
                    cap[q] = __ldcg(g.bf + j);
                    v[q] = __ldg(g.in_col + k);
                } else {
                    cap[q] = __ldcg(g.cf + k);
                    v[q] = __ldg(g.col + k);
                }
            }
            if (rem > 0 && r0 + q < rounds && base < e) scanned += (e - base < W) ? (e - base) : W;
        }
#pragma unroll
        for (int q = 0; q < kIlp; ++q)
            if (cap[q] > 0) hv[q] = __ldcg(P.st.h + v[q]);
#pragma unroll
        for (int q = 0; q < kIlp; ++q) {
            const long long k = b + (long long)(r0 + q) * W + sl;
            long long amt = (cap[q] > 0 && hv[q] < hu && rem > 0) ? (long long)cap[q] : 0;
            long long incl = seg_incl_scan<W>(amt, sl);
            long long tot = __shfl_sync(kFull, incl, W - 1, W);
            long long d = rem - (incl - amt);
            d = d < 0 ? 0 : (d > amt ? amt : d);
            if (d > 0) {
                mp_push<L>(P, u, k, in, v[q], (int)d);
                ++npush;
            }
            if ((long long)cap[q] - d > 0 && hv[q] < hres) hres = hv[q];
            rem -= tot < rem ? tot : rem;
        }
    }
}

template <int L, int W>
__device__ void mp_tile(Ctx &c, int u, int sl, bool phase1, int hcap)
{
    const Params &P = c.P;
    const GraphDev &g = P.g;
    long long ob = 0, oe = 0, ib = 0, ie = 0;
    int ro = 0, ri = 0;
    long long E = 0;
    int hu = 0;
    if (u >= 0) {
        ob = __ldg(g.off + u);
        oe = __ldg(g.off + u + 1);
        ro = (int)((oe - ob + W - 1) / W);
        if (L == kRCSR) {
            ib = __ldg(g.in_off + u);
            ie = __ldg(g.in_off + u + 1);
            ri = (int)((ie - ib + W - 1) / W);
        }
        if (sl == 0) {
            E = __ldcg(P.st.e + u);
            hu = __ldcg(P.st.h + u);
        }
    }
    E = __shfl_sync(kFull, E, 0, W);
    hu = __shfl_sync(kFull, hu, 0, W);
    ro = __reduce_max_sync(kFull, ro);
    if (L == kRCSR) ri = __reduce_max_sync(kFull, ri);
    long long rem = E;
    int hres = 0x7fffffff, npush = 0;
    long long scanned = 0;
    mp_list<L, W>(c, u, ob, oe, ro, false, sl, hu, rem, hres, npush, scanned);
    if (L == kRCSR) mp_list<L, W>(c, u, ib, ie, ri, true, sl, hu, rem, hres, npush, scanned);
    hres = seg_min_int<W>(hres);
    npush = seg_sum_int<W>(npush);
    if (u >= 0 && sl == 0) {
        const long long D = E - rem;
        if (D > 0) atomicAdd((u64 *)(P.st.e + u), (u64)(-D));
        if (npush) atomicAdd((unsigned long long *)&c.sm.stats[kStatPushes], (u64)npush);
        atomicAdd((unsigned long long *)&c.sm.stats[kStatArcs], (u64)scanned);
        if (rem > 0) {
            relabel_to(c, u, hu, hres == 0x7fffffff ? hcap : hres + 1, phase1, hcap);
            touch_mark(P.st, u);
        }
    }
}

// Take the next hub chunk of generation (s3, set): warp-uniform result.
// Chunk ids are reserved in batches (one atomic on the generation's counter
// per `WGrab::batch` chunks), so that hundreds of thousands of chunks per
// pass do not all meet on one counter.
// A warp's chunks come in runs of consecutive ids, which mostly belong to
// one hub: the hub last looked up (queue position `lo`, chunk ids [s0, s1))
// and its row (vertex u, BCSR/RCSR out row at ob of dout entries, RCSR in
// row at ib of din entries) are kept, so that the next chunk of the same
// hub costs no lookup.
struct WGrab {
    unsigned next, end, batch;
    unsigned lo, s0, s1;
    int u;
    long long ob, dout, ib, din;
    __device__ WGrab(unsigned nchunks, unsigned nwarps)
        : next(0), end(0), batch(nchunks / (8u * nwarps) + 1u), lo(0), s0(0), s1(0), u(0), ob(0), dout(0), ib(0),
          din(0) {}
};

template <int L>
__device__ __forceinline__ bool grab_wchunk(Ctx &c, int s3, int set, unsigned nh, unsigned nchunks, WGrab &gb,
                                            unsigned &pos, unsigned &j, unsigned &nch)
{
    if (nchunks <= c.nblk * kWarps) {
        // no more chunks than warps: warp gw takes chunk gw, without an atomic
        const unsigned gw = c.bid * kWarps + (threadIdx.x >> 5);
        if (gb.end != 0 || gw >= nchunks) return false;
        gb.end = 1;
        gb.next = gw;
    } else if (gb.next >= gb.end) {
        unsigned b = 0;
        if ((threadIdx.x & 31) == 0) b = atomicAdd(&c.P.st.ctl->q_grab[s3], gb.batch);
        b = __shfl_sync(kFull, b, 0);
        gb.next = b;
        gb.end = b + gb.batch < nchunks ? b + gb.batch : nchunks;
    }
    if (gb.next >= nchunks) return false;
    const unsigned id = gb.next++;
    if (!(id >= gb.s0 && id < gb.s1)) {  // another hub: look it up and load its row bounds
        unsigned lo = 0, s0 = 0, s1 = 0;
        if ((threadIdx.x & 31) == 0) {
            const unsigned *start = c.P.st.hub_start[set];
            lo = __ldcg(c.P.st.hub_chunk[set] + id);  // start[lo] <= id < start[lo + 1]
            s0 = __ldcg(start + lo);
            s1 = lo + 1 < nh ? __ldcg(start + lo + 1) : nchunks;
        }
        gb.lo = __shfl_sync(kFull, lo, 0);
        gb.s0 = __shfl_sync(kFull, s0, 0);
        gb.s1 = __shfl_sync(kFull, s1, 0);
        const GraphDev &g = c.P.g;
        gb.u = __ldcg(c.P.st.q[set][2] + gb.lo);
        gb.ob = __ldg(g.off + gb.u);
        gb.dout = __ldg(g.off + gb.u + 1) - gb.ob;
        if (L == kRCSR) {
            gb.ib = __ldg(g.in_off + gb.u);
            gb.din = __ldg(g.in_off + gb.u + 1) - gb.ib;
        }
    }
    pos = gb.lo;
    j = id - gb.s0;
    nch = gb.s1 - gb.s0;
    return true;
}

// Rows of the warp class, taken dynamically by warps in batches of `batch`
// (one atomic per batch): the next row index for the calling warp, or
// `count` when none is left.  With no more rows than warps (nwarps), warp gw
// takes row gw, without an atomic: thousands of warps meeting on one counter
// would cost more than the few rows.  Warp-uniform; next = end = 0 at first.
__device__ __forceinline__ unsigned grab_rows(unsigned *ctr, unsigned count, unsigned batch, unsigned &next,
                                              unsigned &end, unsigned gw, unsigned nwarps)
{
    if (count <= nwarps) {
        const unsigned r = end == 0 && gw < count ? gw : count;
        end = 1;
        return r;
    }
    if (next >= end) {
        unsigned b = 0;
        if ((threadIdx.x & 31) == 0) b = atomicAdd(ctr, batch);
        b = __shfl_sync(kFull, b, 0);
        next = b;
        end = b + batch < count ? b + batch : count;
        if (b >= count) return count;
    }
    return next++;
}

// Starts the copies of this lane's 8 entries of hub chunk (pos, j) into the
// stage `buf` (neighbour ids at lane * 8, capacities at kWChunk + lane * 8);
// false (nothing copied) where pr_wchunk would not read them as vectors.
template <int L>
__device__ __forceinline__ bool stage_wchunk(Ctx &c, int set, unsigned pos, unsigned j, int *buf)
{
    constexpr int kPer = kWChunk / 32;
    const GraphDev &g = c.P.g;
    const int lane = threadIdx.x & 31;
    const int u = __ldcg(c.P.st.q[set][2] + pos);
    const long long ob = __ldg(g.off + u);
    const long long a0 = (ob & ~3LL) + (long long)j * kWChunk + (long long)lane * kPer;
    const bool ok = L == kBCSR && a0 >= 0 && a0 + kPer <= g.slots &&
                    ((reinterpret_cast<uintptr_t>(g.col) | reinterpret_cast<uintptr_t>(g.cf)) & 15) == 0;
    if (ok) {
#pragma unroll
        for (int q = 0; q < kPer / 4; ++q) {
            cp_async16(buf + lane * kPer + 4 * q, g.col + a0 + 4 * q);
            cp_async16(buf + kWChunk + lane * kPer + 4 * q, g.cf + a0 + 4 * q);
        }
    }
    return ok;
}

// One chunk of a hub's residual list (kWChunk entries), processed by one
// warp: lane l holds the 8 consecutive entries 8l .. 8l + 7 of the chunk (in
// BCSR read as two aligned 16-byte vectors of col and of cf; the chunk starts
// `lead` slots before the row, entries outside the row are masked).
// Multi-push: the warp sums the capacity of its admissible entries, takes up
// to that much of the hub's remaining excess with a compare-and-swap on the
// hub's budget, and spreads what it took over its admissible entries in slot
// order (one warp scan of the lanes' sums).  Single push: the chunk's minimum
// (height, row index) key.  The last chunk of the hub to finish lowers e(u)
// by what all chunks pushed and relabels u when excess is left (or applies
// the single push/relabel).
template <int L>
__device__ void pr_wchunk(Ctx &c, int set, unsigned pos, unsigned j, unsigned nch, bool phase1, int hcap,
                          const int *staged = nullptr, const WGrab *gb = nullptr)
{
    constexpr int kPer = kWChunk / 32;
    const Params &P = c.P;
    const GraphDev &g = P.g;
    const int lane = threadIdx.x & 31;
    // the hub and its row: from the grabber's cache (the chunk's own hub) or loaded
    const int u = gb ? gb->u : __ldcg(P.st.q[set][2] + pos);
    const long long ob = gb ? gb->ob : __ldg(g.off + u);
    const long long dout = gb ? gb->dout : __ldg(g.off + u + 1) - ob;
    long long ib = 0, din = 0;
    if (L == kRCSR) {
        ib = gb ? gb->ib : __ldg(g.in_off + u);
        din = gb ? gb->din : __ldg(g.in_off + u + 1) - ib;
    }
    const long long deg = dout + din;
    const int lead = L == kBCSR ? (int)(ob & 3) : 0;
    const long long r0 = (long long)j * kWChunk - lead + (long long)lane * kPer;  // row index of entry 0
    const int hu = __ldcg(P.st.h + u);
    bool spent = false;
    if (P.multi_push) spent = __ldcg(P.st.hub_rem[set] + pos) == 0;
    int capv[kPer], vv[kPer], hvv[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        capv[i] = 0;
        vv[i] = 0;
        hvv[i] = 0x7fffffff;
    }
    if (!spent) {
        const long long a0 = ob + r0;  // BCSR: absolute slot of entry 0, a multiple of 4
        const bool vec = L == kBCSR && a0 >= 0 && a0 + kPer <= g.slots &&
                         ((reinterpret_cast<uintptr_t>(g.col) | reinterpret_cast<uintptr_t>(g.cf)) & 15) == 0;
        if (vec) {
            // this lane's entries: from its stage (copied while the warp worked on
            // the previous chunk), else from global memory
            const int4 *sc = staged ? reinterpret_cast<const int4 *>(staged + lane * kPer) : nullptr;
            const int4 *sf = staged ? reinterpret_cast<const int4 *>(staged + kWChunk + lane * kPer) : nullptr;
#pragma unroll
            for (int q = 0; q < kPer / 4; ++q) {
                const int4 cv = sc ? sc[q] : __ldg(reinterpret_cast<const int4 *>(g.col + a0) + q);
                const int4 fv = sf ? sf[q] : __ldcg(reinterpret_cast<const int4 *>(g.cf + a0) + q);
                vv[4 * q] = cv.x; vv[4 * q + 1] = cv.y; vv[4 * q + 2] = cv.z; vv[4 * q + 3] = cv.w;
                capv[4 * q] = fv.x; capv[4 * q + 1] = fv.y; capv[4 * q + 2] = fv.z; capv[4 * q + 3] = fv.w;
            }
#pragma unroll
            for (int i = 0; i < kPer; ++i)
                if (r0 + i < 0 || r0 + i >= deg) capv[i] = 0;  // outside the row
#pragma unroll
            for (int i = 0; i < kPer; ++i)
                if (capv[i] > 0) hvv[i] = __ldcg(P.st.h + vv[i]);
        } else {
#pragma unroll
            for (int i = 0; i < kPer; ++i) {
                const long long r = r0 + i;
                if (r >= 0 && r < deg) {
                    bool in;
                    const long long k = row_slot<L>(ob, dout, ib, r, in);
                    mp_load<L>(P, k, in, capv[i], vv[i], hvv[i]);
                }
            }
        }
    }
    if (lane == 0 && !spent) {
        const long long lo = (long long)j * kWChunk - lead, hi = lo + kWChunk;
        const long long n_in = (hi < deg ? hi : deg) - (lo > 0 ? lo : 0);
        if (n_in > 0) atomicAdd((unsigned long long *)&c.sm.stats[kStatArcs], (u64)n_in);
    }
    if (!P.multi_push) {
        u64 best = kNoKey;
#pragma unroll
        for (int i = 0; i < kPer; ++i)
            if (capv[i] > 0) best = umin64(best, make_key(hvv[i], (unsigned)(r0 + i)));
        best = tile_min<32>(best);
        if (lane == 0 && best != kNoKey) atomicMin(P.st.hub_aux[set] + pos, best);
    } else {
        long long asum = 0;
#pragma unroll
        for (int i = 0; i < kPer; ++i)
            if (capv[i] > 0 && hvv[i] < hu) asum += capv[i];
        const long long incl = seg_incl_scan<32>(asum, lane);
        const long long tot = __shfl_sync(kFull, incl, 31);
        long long take = 0;
        if (lane == 0 && tot > 0) {
            long long *rp = P.st.hub_rem[set] + pos;
            long long r = __ldcg(rp);
            for (int tries = 0; tries < (1 << 20) && r > 0; ++tries) {
                const long long t = r < tot ? r : tot;
                const long long prev = (long long)atomicCAS((u64 *)rp, (u64)r, (u64)(r - t));
                if (prev == r) {
                    take = t;
                    break;
                }
                r = prev;
            }
        }
        take = __shfl_sync(kFull, take, 0);
        long long budget = take - (incl - asum);
        budget = budget < 0 ? 0 : (budget > asum ? asum : budget);
        int npush = 0, hres = 0x7fffffff;
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            int cap = capv[i];
            if (cap > 0 && hvv[i] < hu && budget > 0) {
                bool in = false;
                const long long k = row_slot<L>(ob, dout, ib, r0 + i, in);
                const int d = (int)(budget < cap ? budget : cap);
                mp_push<L>(P, u, k, in, vv[i], d);
                budget -= d;
                cap -= d;
                ++npush;
            }
            if (cap > 0 && hvv[i] < hres) hres = hvv[i];
        }
        hres = seg_min_int<32>(hres);
        npush = seg_sum_int<32>(npush);
        if (lane == 0) {
            if (hres != 0x7fffffff) atomicMin(P.st.hub_aux[set] + pos, (u64)(unsigned)hres << 32);
            if (npush) atomicAdd((unsigned long long *)&c.sm.stats[kStatPushes], (u64)npush);
        }
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) {
        const unsigned done = atomicAdd(P.st.hub_done[set] + pos, 1u);
        if (done + 1 == nch) {
            __threadfence();
            const u64 key = __ldcg(P.st.hub_aux[set] + pos);
            if (!P.multi_push) {
                apply_op<L>(c, u, key, phase1, hcap);
            } else {
                const long long rem = __ldcg(P.st.hub_rem[set] + pos);
                const long long D = __ldcg(P.st.hub_e0[set] + pos) - rem;
                if (D > 0) atomicAdd((u64 *)(P.st.e + u), (u64)(-D));
                if (rem > 0) {
                    relabel_to(c, u, hu, key == kNoKey ? hcap : (int)(key >> 32) + 1, phase1, hcap);
                    touch_mark(P.st, u);
                }
            }
        }
    }
    __syncwarp();
}

// Consume the AVQ of generation `gen` (step 3 of an iteration).
// Per-warp busy time (the per-warp execution-time record of §4.3, taken by
// the warp's first lane): from the start of a push-relabel pass to the end of
// the warp's share of it, summed over the passes of a solve.
__device__ __forceinline__ u64 warp_clock(const Params &P)
{
    return P.warp_ns && (threadIdx.x & 31) == 0 ? global_ns() : 0ull;
}

__device__ __forceinline__ void warp_clock_add(const Ctx &c, u64 t0)
{
    if (c.P.warp_ns && (threadIdx.x & 31) == 0)
        c.P.warp_ns[(u64)c.bid * kWarps + (threadIdx.x >> 5)] += global_ns() - t0;
}

template <int L, int SW>
__device__ void pr_process(Ctx &c, bool phase1, int hcap)
{
    const Params &P = c.P;
    Ctl *ctl = P.st.ctl;
    const int gen = c.gen, s3 = gen % 3, set = gen & 1;
    const u64 wt0 = warp_clock(P);
    reset_rotating(c, gen);
    reset_local_slot(c, gen);
    const unsigned c0 = __ldcg(&ctl->q_count[s3][0]);
    const unsigned c1 = __ldcg(&ctl->q_count[s3][1]);
    const int lane = threadIdx.x & 31;
    const unsigned gwarp = c.bid * kWarps + (threadIdx.x >> 5);
    const unsigned nwarps = c.nblk * kWarps;
    {
        // warp-class rows: taken dynamically, in batches (their lengths vary
        // from small_max to warp_max entries)
        const int *q1 = P.st.q[set][1];
        const unsigned batch = c1 / (8u * nwarps) + 1u;
        unsigned next = 0, end = 0;
        for (;;) {
            const unsigned i = grab_rows(&ctl->q_grab_w[s3], c1, batch, next, end, gwarp, nwarps);
            if (i >= c1) break;
            if (P.multi_push) mp_tile<L, 32>(c, __ldcg(q1 + i), lane, phase1, hcap);
            else pr_tile<L, 32>(c, __ldcg(q1 + i), lane, phase1, hcap);
        }
    }
    {
        constexpr unsigned TPW = 32 / SW;
        const unsigned gt0 = gwarp * TPW, ntiles = nwarps * TPW;
        const int *q0 = P.st.q[set][0];
        if (c0 > gt0) {
            const unsigned rounds = (c0 - gt0 + ntiles - 1) / ntiles;
            const unsigned sub = lane / SW, sl = lane % SW;
            for (unsigned r = 0; r < rounds; ++r) {
                unsigned i = gt0 + sub + r * ntiles;
                int u = i < c0 ? __ldcg(q0 + i) : -1;
                if (P.multi_push) mp_tile<L, SW>(c, u, sl, phase1, hcap);
                else pr_tile<L, SW>(c, u, sl, phase1, hcap);
            }
        }
    }
    // hub rows last: chunks taken dynamically, one warp each, fill the tail
    {
        const u64 hp = __ldcg(&ctl->hub_pack[s3]);
        const unsigned nh = (unsigned)(hp >> 40), nchunks = (unsigned)(hp & kChunkMask);
        unsigned pos, j, nch;
        if (nchunks) {
            if (L == kBCSR && c.stage) {
                // Staged: the warp takes its next chunk before working on the
                // current one and copies the next chunk's entries into its
                // other buffer meanwhile.
                int *wb = c.stage + (threadIdx.x >> 5) * kStageInts;
                WGrab gb(nchunks, c.nblk * kWarps);
                bool have = grab_wchunk<L>(c, s3, set, nh, nchunks, gb, pos, j, nch);
                bool st = have && stage_wchunk<L>(c, set, pos, j, wb);
                cp_async_commit();
                int b = 0;
                while (have) {
                    unsigned pos2, j2, nch2;
                    const bool have2 = grab_wchunk<L>(c, s3, set, nh, nchunks, gb, pos2, j2, nch2);
                    const bool st2 = have2 && stage_wchunk<L>(c, set, pos2, j2, wb + (b ^ 1) * 2 * kWChunk);
                    cp_async_commit();
                    cp_async_wait<1>();  // the current chunk's copies are done
                    pr_wchunk<L>(c, set, pos, j, nch, phase1, hcap, st ? wb + b * 2 * kWChunk : nullptr);
                    pos = pos2;
                    j = j2;
                    nch = nch2;
                    have = have2;
                    st = st2;
                    b ^= 1;
                }
                cp_async_wait<0>();
            } else {
                WGrab gb(nchunks, c.nblk * kWarps);
                while (grab_wchunk<L>(c, s3, set, nh, nchunks, gb, pos, j, nch))
                    pr_wchunk<L>(c, set, pos, j, nch, phase1, hcap, nullptr, &gb);
            }
        }
    }
    warp_clock_add(c, wt0);
}

// Block-local pass for a small AVQ (avq_incremental = 2): every block takes
// the candidate-bitmap words w = bid, bid + nblk, ... (so that a run of
// consecutive vertices spreads over the blocks), clears them atomically,
// ranks the marked vertices that are active by tile class in shared memory
// and processes them itself: the compaction and the pass share one grid
// barrier.  Every vertex belongs to one word and every word to one block,
// so a vertex is processed at most once per pass, by its word's block.  A
// push may land in a word already cleared in this pass (its target waits
// for the next pass), or in one not yet cleared (its target may be
// processed in this pass, with the excess that has arrived).  Hubs, and
// candidates beyond the block's staging, stay marked and make the next
// iteration a full one.  The team's active count and the deferral flag go
// to ctl->local_active / local_defer, slot gen % 3.
template <int L, int SW>
__device__ void pr_local(Ctx &c, bool phase1, int hcap)
{
    const Params &P = c.P;
    const GraphDev &g = P.g;
    const int s = g.s, t = g.t;
    const int gen = c.gen, s3 = gen % 3;
    const u64 wt0 = warp_clock(P);
    reset_local_slot(c, gen);  // (the rotating queue counters are cleared after the pass: see iterate())
    const long long nwords = ((long long)g.n + 31) >> 5;
    int *cand = c.sm.qbuf[0];
    int *smallq = c.sm.qbuf[1];
    int *warpq = c.sm.qbuf[2];
    __syncthreads();  // qcnt is zero between passes; every thread sees it before the counts grow
    bool defer = false;
    long long nc = 0;
    for (long long w = c.bid + (long long)threadIdx.x * c.nblk; w < nwords; w += (long long)kBlock * c.nblk) {
        unsigned bits = __ldcg(P.st.touch + w);
        if (!bits) continue;
        bits = atomicExch(P.st.touch + w, 0u);
        while (bits) {
            const unsigned pos = atomicAdd(&c.sm.qcnt[0], 1u);
            if (pos >= (unsigned)kQueueCap) {  // staging full: leave the rest marked
                atomicOr(P.st.touch + w, bits);
                defer = true;
                break;
            }
            cand[pos] = (int)(w * 32 + (__ffs(bits) - 1));
            bits &= bits - 1;
            ++nc;
        }
    }
    __syncthreads();
    const unsigned ncand = c.sm.qcnt[0] < (unsigned)kQueueCap ? c.sm.qcnt[0] : (unsigned)kQueueCap;
    long long nact = 0;
    for (unsigned j = threadIdx.x; j < ncand; j += kBlock) {
        const int v = cand[j];
        if (v == s || v == t || __ldcg(P.st.h + v) >= hcap || __ldcg(P.st.e + v) <= 0) continue;
        const int cls = classify(P, degree<L>(g, v));
        if (cls == 2) {  // a hub: chunked over the whole team by a full pass
            atomicOr(P.st.touch + (v >> 5), 1u << (v & 31));
            defer = true;
            continue;
        }
        ++nact;
        if (cls == 0) smallq[atomicAdd(&c.sm.qcnt[1], 1u)] = v;
        else warpq[atomicAdd(&c.sm.qcnt[2], 1u)] = v;
    }
    __syncthreads();
    const unsigned nsmall = c.sm.qcnt[1], nwarp = c.sm.qcnt[2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (unsigned i = warp; i < nwarp; i += kWarps) {
        if (P.multi_push) mp_tile<L, 32>(c, warpq[i], lane, phase1, hcap);
        else pr_tile<L, 32>(c, warpq[i], lane, phase1, hcap);
    }
    constexpr unsigned TPW = 32 / SW;
    for (unsigned base = warp * TPW; base < nsmall; base += kWarps * TPW) {
        const unsigned idx = base + lane / SW;
        const int u = idx < nsmall ? smallq[idx] : -1;
        if (P.multi_push) mp_tile<L, SW>(c, u, lane % SW, phase1, hcap);
        else pr_tile<L, SW>(c, u, lane % SW, phase1, hcap);
    }
    const long long ba = block_sum(c, nact);
    const long long bc = block_sum(c, nc);
    const int bd = __syncthreads_or(defer);
    if (threadIdx.x == 0) {
        if (ba) {
            atomicAdd(&P.st.ctl->local_active[s3], (unsigned)ba);
            atomicAdd((unsigned long long *)&c.sm.stats[kStatActive], (u64)ba);
        }
        if (bc) atomicAdd((unsigned long long *)&c.sm.stats[kStatAvqCand], (u64)bc);
        if (bd) atomicExch(&P.st.ctl->local_defer[s3], 1);
        if (c.bid == 0) atomicAdd((unsigned long long *)&c.sm.stats[kStatAvqInc], 1ull);
    }
    if (threadIdx.x < kClasses) c.sm.qcnt[threadIdx.x] = 0;
    __syncthreads();
    warp_clock_add(c, wt0);
}

// One thread-centric pass (the lock-free algorithm of Alg. 1 as the paper's
// TC baseline runs it): every thread owns vertices tid, tid + grid, ...,
// checks each for activity itself, and scans an active vertex's whole
// residual list alone (a tile of one lane), then pushes or relabels.  No AVQ
// and no degree classes: the warp waits for its longest row.  The pass
// counts the active vertices it found (queue counter of class 0, so that an
// empty pass ends the iterations), and applies a pending gap as the AVQ
// compaction does, to the vertices each thread owns.
template <int L>
__device__ void tc_process(Ctx &c, bool phase1, int hcap)
{
    const Params &P = c.P;
    const GraphDev &g = P.g;
    const int n = g.n, s = g.s, t = g.t;
    const int gen = c.gen, s3 = gen % 3;
    const u64 wt0 = warp_clock(P);
    // The rotating counters of generation gen - 1 (whose gap candidate is
    // read here) are cleared after the pass's grid barrier, in iterate().
    int gap = kUnvisited;
    if (phase1 && P.gap) {
        const int cand = __ldcg(&P.st.ctl->gap_level[(gen + 2) % 3]);
        if (cand < n && __ldcg(P.st.count + cand) == 0) gap = cand;
    }
    const long long stride = (long long)c.nblk * kBlock;
    const long long rounds = ((long long)n + stride - 1) / stride;  // the same for every thread
    long long nact = 0;
    for (long long r = 0; r < rounds; ++r) {
        const long long v = r * stride + (long long)c.bid * kBlock + threadIdx.x;
        int u = -1;
        if (v < n && v != s && v != t) {
            int hv = __ldcg(P.st.h + v);
            if (gap != kUnvisited && hv > gap && hv < n) {
                hv = n;
                __stcg(P.st.h + v, n);
            }
            if (hv < hcap && __ldcg(P.st.e + v) > 0) u = (int)v;
        }
        nact += u >= 0;
        if (P.multi_push) mp_tile<L, 1>(c, u, 0, phase1, hcap);
        else pr_tile<L, 1>(c, u, 0, phase1, hcap);
    }
    const long long bn = block_sum(c, nact);
    if (threadIdx.x == 0 && bn) {
        atomicAdd(&P.st.ctl->q_count[s3][0], (unsigned)bn);
        atomicAdd((unsigned long long *)&c.sm.stats[kStatActive], (u64)bn);
    }
    if (c.bid == 0 && threadIdx.x == 0 && gap != kUnvisited)
        atomicAdd((unsigned long long *)&c.sm.stats[kStatGaps], 1ull);
    warp_clock_add(c, wt0);
}

// Incremental compaction: between two global relabels a vertex can turn
// active only by receiving a push (its height only grows, its excess only
// grows through pushes), and an active vertex stays active only if its owner
// left excess after its pass; both mark the vertex in the candidate bitmap.
// So the AVQ is the set of marked vertices with e > 0 and h below the cap.
// Warps take 32 bitmap words (1,024 vertices) at a time and clear them; the
// marked vertices of the 32 words are dealt to the lanes 32 at a time (a
// warp scan of the words' bit counts; each lane finds the word and the bit
// of its candidate), ballots rank the active ones per tile class, and one
// atomic per class and round places them.
template <int L>
__device__ void build_avq_inc(Ctx &c, int hcap)
{
    const Params &P = c.P;
    const GraphDev &g = P.g;
    const int s = g.s, t = g.t;
    const int gen = c.gen, s3 = gen % 3, set = gen & 1;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const long long nwords = ((long long)g.n + 31) >> 5;
    const long long gwarp = (long long)c.bid * kWarps + (threadIdx.x >> 5);
    const long long nwarps = (long long)c.nblk * kWarps;
    long long nact = 0;
    for (long long w0 = gwarp * 32; w0 < nwords; w0 += nwarps * 32) {
        const long long w = w0 + lane;
        const unsigned bits = w < nwords ? __ldcg(P.st.touch + w) : 0u;
        if (bits) __stcg(P.st.touch + w, 0u);
        const unsigned cnt = __popc(bits);
        unsigned incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const unsigned total = __shfl_sync(kFull, incl, 31);
        if (lane == 0 && total) atomicAdd((unsigned long long *)&c.sm.stats[kStatAvqCand], (u64)total);
        for (unsigned r0 = 0; r0 < total; r0 += 32) {
            const unsigned k = r0 + lane;  // this lane's candidate: the k-th marked vertex of the words
            unsigned src = 0;              // its word: lanes whose inclusive count is <= k
#pragma unroll
            for (unsigned b = 16; b > 0; b >>= 1) {
                const unsigned x = __shfl_sync(kFull, incl, src + b - 1);
                if (x <= k) src += b;
            }
            const unsigned sl = src < 32 ? src : 31;
            unsigned word = __shfl_sync(kFull, bits, sl);
            const unsigned before = __shfl_sync(kFull, incl, sl) - __shfl_sync(kFull, cnt, sl);
            int v = -1;
            if (k < total) {
                for (unsigned i = before; i < k; ++i) word &= word - 1;  // drop the bits before it
                v = (int)((w0 + sl) * 32 + (__ffs(word) - 1));
            }
            long long ev = 0, d = 0;
            int cls = -1;
            if (v >= 0 && v != s && v != t && __ldcg(P.st.h + v) < hcap) {
                ev = __ldcg(P.st.e + v);
                if (ev > 0) {
                    d = degree<L>(g, v);
                    cls = classify(P, d);
                    ++nact;
                }
            }
            warp_hub_append<L>(c, s3, set, cls == 2, v, d, ev);
            const unsigned m0 = __ballot_sync(kFull, cls == 0), m1 = __ballot_sync(kFull, cls == 1);
            unsigned b0 = 0, b1 = 0;
            if (lane == 0 && m0) b0 = atomicAdd(&P.st.ctl->q_count[s3][0], (unsigned)__popc(m0));
            if (lane == 0 && m1) b1 = atomicAdd(&P.st.ctl->q_count[s3][1], (unsigned)__popc(m1));
            b0 = __shfl_sync(kFull, b0, 0);
            b1 = __shfl_sync(kFull, b1, 0);
            if (cls == 0) P.st.q[set][0][b0 + __popc(m0 & lt)] = v;
            if (cls == 1) P.st.q[set][1][b1 + __popc(m1 & lt)] = v;
        }
    }
    if (nact) atomicAdd((unsigned long long *)&c.sm.stats[kStatActive], (u64)nact);
    if (c.bid == 0 && threadIdx.x == 0) atomicAdd((unsigned long long *)&c.sm.stats[kStatAvqInc], 1ull);
}

// Step 1 of an iteration: build the AVQ of generation `gen`.  `first`: the
// first compaction after a global relabel, which moved heights both ways, so
// every vertex is scanned (and the candidate bitmap cleared); later ones use
// the bitmap unless a gap must be applied (it lifts unmarked vertices too).
template <int L>
__device__ void build_avq(Ctx &c, bool phase1, int hcap, bool first)
{
    const Params &P = c.P;
    const GraphDev &g = P.g;
    const int n = g.n, s = g.s, t = g.t;
    const int gen = c.gen, s3 = gen % 3, set = gen & 1;
    // Gap check at this quiescent point (phase 1 only).
    int gap = kUnvisited;
    if (phase1 && P.gap) {
        int cand = __ldcg(&P.st.ctl->gap_level[(gen + 2) % 3]);
        if (cand < n && __ldcg(P.st.count + cand) == 0) gap = cand;
    }
    if (P.st.touch) {
        if (!first && gap == kUnvisited) {
            build_avq_inc<L>(c, hcap);
            return;
        }
        const long long nwords = ((long long)n + 31) >> 5;
        for (long long w = (long long)c.bid * kBlock + threadIdx.x; w < nwords; w += (long long)c.nblk * kBlock)
            __stcg(P.st.touch + w, 0u);
    }
    if (c.bid == 0 && threadIdx.x == 0) atomicAdd((unsigned long long *)&c.sm.stats[kStatAvqFull], 1ull);
    // kAvqVerts vertices per thread per step, their loads issued together
    // (heights, then excesses, then row offsets of the active ones).  The
    // blocks take the steps of kBlock * kAvqVerts vertices in turn, so that a
    // run of long rows (a renumbered graph puts its hubs first) is spread
    // over many blocks.
    constexpr int kAvqVerts = 4;
    constexpr long long kStep = (long long)kBlock * kAvqVerts;
    long long nact = 0;
    const long long v1 = n;
    for (long long base = (long long)c.bid * kStep; base < n; base += (long long)c.nblk * kStep) {
        int hv[kAvqVerts];
        long long ev[kAvqVerts], d[kAvqVerts];
#pragma unroll
        for (int i = 0; i < kAvqVerts; ++i) {
            const long long v = base + (long long)i * kBlock + threadIdx.x;
            hv[i] = v < v1 ? __ldcg(P.st.h + v) : hcap;
        }
#pragma unroll
        for (int i = 0; i < kAvqVerts; ++i) {
            const long long v = base + (long long)i * kBlock + threadIdx.x;
            if (v < v1 && gap != kUnvisited && hv[i] > gap && hv[i] < n && v != s) {
                hv[i] = n;
                __stcg(P.st.h + v, n);
            }
            ev[i] = (v < v1 && v != s && v != t && hv[i] < hcap) ? __ldcg(P.st.e + v) : 0;
        }
#pragma unroll
        for (int i = 0; i < kAvqVerts; ++i) {
            const long long v = base + (long long)i * kBlock + threadIdx.x;
            d[i] = ev[i] > 0 ? degree<L>(g, (int)v) : 0;
        }
        // Compaction of the active vertices of classes 0 and 1: per round a
        // warp ballot of each class gives every lane its rank in the warp; a
        // block prefix over the warps' counts and one global atomic per class
        // give the block's range in the queue (Alg. 2's atomic append,
        // aggregated over 1024 vertices).  Hubs take their chunk ids from the
        // hub counter.
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const unsigned lt = (1u << lane) - 1u;
        int cls[kAvqVerts];
        unsigned m0[kAvqVerts], m1[kAvqVerts], w0 = 0, w1 = 0;
#pragma unroll
        for (int i = 0; i < kAvqVerts; ++i) {
            cls[i] = -1;
            if (ev[i] > 0) {
                cls[i] = classify(P, d[i]);
                ++nact;
            }
            const int v = (int)(base + (long long)i * kBlock + threadIdx.x);
            warp_hub_append<L>(c, s3, set, cls[i] == 2, v, d[i], ev[i]);
            m0[i] = __ballot_sync(kFull, cls[i] == 0);
            m1[i] = __ballot_sync(kFull, cls[i] == 1);
            w0 += __popc(m0[i]);
            w1 += __popc(m1[i]);
        }
        if (lane == 0) {
            c.sm.wcnt[0][warp] = w0;
            c.sm.wcnt[1][warp] = w1;
        }
        __syncthreads();
        if (threadIdx.x < 2) {
            unsigned tot = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) tot += c.sm.wcnt[threadIdx.x][w];
            c.sm.gbase[threadIdx.x] = tot ? atomicAdd(&P.st.ctl->q_count[s3][threadIdx.x], tot) : 0u;
        }
        __syncthreads();
        unsigned b0 = c.sm.gbase[0], b1 = c.sm.gbase[1];
        for (int w = 0; w < warp; ++w) {
            b0 += c.sm.wcnt[0][w];
            b1 += c.sm.wcnt[1][w];
        }
#pragma unroll
        for (int i = 0; i < kAvqVerts; ++i) {
            const int v = (int)(base + (long long)i * kBlock + threadIdx.x);
            if (cls[i] == 0) P.st.q[set][0][b0 + __popc(m0[i] & lt)] = v;
            if (cls[i] == 1) P.st.q[set][1][b1 + __popc(m1[i] & lt)] = v;
            b0 += __popc(m0[i]);
            b1 += __popc(m1[i]);
        }
        __syncthreads();  // the counts are read before the next step writes them
    }
    if (nact) atomicAdd((unsigned long long *)&c.sm.stats[kStatActive], (u64)nact);
    if (c.bid == 0 && threadIdx.x == 0 && gap != kUnvisited)
        atomicAdd((unsigned long long *)&c.sm.stats[kStatGaps], 1ull);
}

// ---------------------------------------------------------------------------
// Level-synchronous BFS (global relabel and cut).
//   kBfsBackward: from `target`, visit v when the residual arc v -> w exists
//                 (w = frontier vertex); h[v] = level value (CAS on kUnvisited)
//   kBfsForward:  from s, visit v when the residual arc w -> v exists; marks in
//                 count[] (CAS 0 -> level value; s holds 1)
// ---------------------------------------------------------------------------
enum { kBfsBackward = 0, kBfsForward = 1 };

template <int L, int DIR>
__device__ __forceinline__ bool residual_to(const Params &P, long long slot, bool in_slot,
                                            int w)
{
    const GraphDev &g = P.g;
    if (L == kBCSR) {
        if (DIR == kBfsForward) return __ldcg(g.cf + slot) > 0;
        if (g.cfb) return __ldcg(g.cfb + slot) > 0;
        long long ra;
        if (P.use_rev) {
            ra = __ldg(g.rev + slot);
        } else {
            int v = __ldg(g.col + slot);
            ra = lower_bound_col(g.col, __ldg(g.off + v), __ldg(g.off + v + 1), w);
        }
        return __ldcg(g.cf + ra) > 0;
    } else {
        if (!in_slot) {  // out slot j of w: arc w -> v
            return DIR == kBfsForward ? __ldcg(g.cf + slot) > 0 : __ldcg(g.bf + slot) > 0;
        }
        unsigned j = __ldg(g.flow_idx + slot);  // in slot of w: arc v -> w is out slot j
        return DIR == kBfsForward ? __ldcg(g.bf + j) > 0 : __ldcg(g.cf + j) > 0;
    }
}

// Queue vertex v (row length d) in the next frontier, after its claim.
template <int L>
__device__ __forceinline__ void bfs_claimed(Ctx &c, int v, long long d, int nset, int n3)
{
    c.fe += d;
    const int cls = classify(c.P, d);
    if (cls == 2) hub_append(c, n3, nset, v, d, false, 0, kWChunk, hub_lead<L>(c.P.g, v));
    else q_append(c, n3, nset, cls, v);
}

// Where the residual capacity that decides a BFS step over entry k of w's
// list lives, and the neighbour v.  Backward: the arc v -> w; forward: w -> v.
template <int L, int DIR>
__device__ __forceinline__ const int *bfs_res_ptr(const Params &P, long long k, bool in, int w, int &v)
{
    const GraphDev &g = P.g;
    if (L == kBCSR) {
        v = __ldg(g.col + k);
        if (DIR == kBfsForward) return g.cf + k;
        if (g.cfb) return g.cfb + k;  // mirrored backward residual, read in place
        if (P.use_rev) return g.cf + __ldg(g.rev + k);
        return g.cf + lower_bound_col(g.col, __ldg(g.off + v), __ldg(g.off + v + 1), w);
    }
    if (!in) {  // out slot k of w: arc w -> v
        v = __ldg(g.col + k);
        return DIR == kBfsForward ? g.cf + k : g.bf + k;
    }
    v = __ldg(g.in_col + k);  // in slot of w: arc v -> w is out slot j
    const unsigned j = __ldg(g.flow_idx + k);
    return DIR == kBfsForward ? g.bf + j : g.cf + j;
}

// Visit up to NB entries at once: every load of a stage is issued before the
// next stage (address, residual, visited mark), then the claims.
template <int L, int DIR, int NB>
__device__ __forceinline__ void bfs_entries(Ctx &c, int w, const long long (&k)[NB], const bool (&in)[NB],
                                            const bool (&ok)[NB], int val, int nset, int n3)
{
    const Params &P = c.P;
    int v[NB];
    const int *rp[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        v[q] = 0;
        rp[q] = nullptr;
        if (ok[q]) rp[q] = bfs_res_ptr<L, DIR>(P, k[q], in[q], w, v[q]);
    }
    bool res[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) res[q] = ok[q] && __ldcg(rp[q]) > 0;
    bool open[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        open[q] = false;
        if (res[q]) open[q] = DIR == kBfsBackward ? __ldcg(P.st.h + v[q]) == kUnvisited
                                                  : __ldcg(P.st.count + v[q]) == 0;
    }
    // Claims of the open entries: all compare-and-swaps first, then the row
    // bounds of the vertices won, then the appends, so that a lane's claims
    // overlap instead of waiting out three round trips each.
    int old[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        old[q] = 1;
        if (open[q]) old[q] = DIR == kBfsBackward ? atomicCAS(P.st.h + v[q], kUnvisited, val)
                                                  : atomicCAS(P.st.count + v[q], 0, val);
    }
    long long d[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        d[q] = -1;
        if (open[q] && old[q] == (DIR == kBfsBackward ? kUnvisited : 0)) d[q] = degree<L>(P.g, v[q]);
    }
#pragma unroll
    for (int q = 0; q < NB; ++q)
        if (d[q] >= 0) bfs_claimed<L>(c, v[q], d[q], nset, n3);
}

// Scan frontier vertex w with `W` lanes starting at lane `sl`.
template <int L, int DIR, int W>
__device__ void bfs_row(Ctx &c, int w, int sl, int val, int nset, int n3)
{
    constexpr int NB = 4;
    const GraphDev &g = c.P.g;
    const long long ob = __ldg(g.off + w), dout = __ldg(g.off + w + 1) - ob;
    long long ib = 0, din = 0;
    if (L == kRCSR) {
        ib = __ldg(g.in_off + w);
        din = __ldg(g.in_off + w + 1) - ib;
    }
    const long long deg = dout + din;
    for (long long r0 = sl; r0 < deg; r0 += (long long)NB * W) {
        long long k[NB];
        bool in[NB], ok[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const long long r = r0 + (long long)q * W;
            ok[q] = r < deg;
            k[q] = row_slot<L>(ob, dout, ib, ok[q] ? r : 0, in[q]);
        }
        bfs_entries<L, DIR, NB>(c, w, k, in, ok, val, nset, n3);
    }
}

// Scan one chunk of kWChunk entries of frontier hub w with one warp (the
// chunk starts `lead` slots before the row, as in the push-relabel pass);
// lane l takes entries l, l + 32, ... so that every load is coalesced, and
// all loads of a stage are issued together.  Returns the row entries of the
// chunk on lane 0 (0 elsewhere).
template <int L, int DIR>
__device__ long long bfs_wchunk(Ctx &c, const WGrab &gb, unsigned j, int val, int nset, int n3)
{
    constexpr int NB = kWChunk / 32;
    const int lane = threadIdx.x & 31;
    const int w = gb.u;  // the chunk's hub and its row, cached by the grabber
    const long long ob = gb.ob, dout = gb.dout;
    long long ib = 0, din = 0;
    if (L == kRCSR) {
        ib = gb.ib;
        din = gb.din;
    }
    const long long deg = dout + din;
    const long long lo = (long long)j * kWChunk - (L == kBCSR ? (ob & 3) : 0);
    long long k[NB];
    bool in[NB], ok[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        const long long r = lo + lane + 32LL * q;
        ok[q] = r >= 0 && r < deg;
        k[q] = row_slot<L>(ob, dout, ib, ok[q] ? r : 0, in[q]);
    }
    bfs_entries<L, DIR, NB>(c, w, k, in, ok, val, nset, n3);
    const long long hi = lo + kWChunk < deg ? lo + kWChunk : deg;
    return lane == 0 && hi > (lo > 0 ? lo : 0) ? hi - (lo > 0 ? lo : 0) : 0;
}


// Consume frontier generation `gen`, produce generation gen + 1.
template <int L, int DIR, int SW>
__device__ void bfs_level(Ctx &c, int val)
{
    const Params &P = c.P;
    Ctl *ctl = P.st.ctl;
    const int gen = c.gen, s3 = gen % 3, set = gen & 1;
    const int n3 = (gen + 1) % 3, nset = (gen + 1) & 1;
    reset_rotating(c, gen);
    const unsigned c0 = __ldcg(&ctl->q_count[s3][0]);
    const unsigned c1 = __ldcg(&ctl->q_count[s3][1]);
    long long scanned = 0;
    const int lane = threadIdx.x & 31;
    const unsigned gwarp = c.bid * kWarps + (threadIdx.x >> 5);
    const unsigned nwarps = c.nblk * kWarps;
    {
        // warp-class rows (up to warp_max entries, of uneven length): taken
        // dynamically, in batches that keep the atomics few
        const int *q1 = P.st.q[set][1];
        const unsigned batch = c1 / (8u * nwarps) + 1u;
        unsigned next = 0, end = 0;
        for (;;) {
            const unsigned i = grab_rows(&ctl->q_grab_w[s3], c1, batch, next, end, gwarp, nwarps);
            if (i >= c1) break;
            const int w = __ldcg(q1 + i);
            bfs_row<L, DIR, 32>(c, w, lane, val, nset, n3);
            if (lane == 0) scanned += degree<L>(P.g, w);
        }
    }
    {
        const int *q0 = P.st.q[set][0];
        const unsigned gt = (c.bid * kBlock + threadIdx.x) / SW;
        const unsigned ntiles = c.nblk * kBlock / SW;
        const int sl = threadIdx.x % SW;
        for (unsigned i = gt; i < c0; i += ntiles) {
            int w = __ldcg(q0 + i);
            bfs_row<L, DIR, SW>(c, w, sl, val, nset, n3);
            if (sl == 0) scanned += degree<L>(P.g, w);
        }
    }
    {
        // hub rows last: 256-entry chunks taken dynamically, one warp each
        const u64 hp = __ldcg(&ctl->hub_pack[s3]);
        const unsigned nh = (unsigned)(hp >> 40), nchunks = (unsigned)(hp & kChunkMask);
        unsigned pos, j, nch;
        if (nchunks) {
            WGrab gb(nchunks, nwarps);
            while (grab_wchunk<L>(c, s3, set, nh, nchunks, gb, pos, j, nch))
                scanned += bfs_wchunk<L, DIR>(c, gb, j, val, nset, n3);
        }
    }
    q_flush(c, n3, nset);
    if (scanned) atomicAdd((unsigned long long *)&c.sm.stats[kStatGrArcs], (u64)scanned);
    const long long bfe = block_sum(c, c.fe);   // the next frontier's entries, for the direction rule
    if (threadIdx.x == 0 && bfe) atomicAdd((u64 *)&P.st.ctl->fedges[n3], (u64)bfe);
    c.fe = 0;
}

// ---------------------------------------------------------------------------
// Bottom-up level of a BFS (direction-optimising BFS, Beamer, Asanovic and
// Patterson, SC 2012).  Instead of scanning the frontier's rows, every
// unvisited vertex v scans its own row for a residual arc into the frontier
// (v -> w for the backward BFS of the global relabel, w -> v for the forward
// BFS of the cut; w in the frontier when its level value is val - 1) and
// stops at the first one.  It visits exactly the vertices a top-down level
// visits, with the same value, so the distances are unchanged; only the
// entries read differ.  Only v's owner writes v's level, so no claim is
// needed.  Rows of up to kBuThread entries are
// scanned by one thread (kBuVerts vertices per thread, 4 entries per step),
// longer rows by a warp, hub rows by a warp for their first kBuHubHead
// entries and by the whole block for the rest.
// ---------------------------------------------------------------------------
constexpr int kBuThread = 32;
constexpr int kBuStep = 4;
constexpr long long kBuHubHead = 4 * 32 * kBuStep;  // hub-row entries a warp scans first

// Over entry k of v's list (neighbour w returned): the residual capacity of
// v -> w (backward BFS) or of w -> v (forward BFS; BCSR without the mirror:
// the reverse slot by index or by binary search in w's row).
template <int L, int DIR>
__device__ __forceinline__ int bu_res(const Params &P, int v, long long k, bool in, int &w)
{
    const GraphDev &g = P.g;
    if (L == kBCSR) {
        w = __ldg(g.col + k);
        if (DIR == kBfsBackward) return __ldcg(g.cf + k);
        if (g.cfb) return __ldcg(g.cfb + k);
        const long long ra = P.use_rev ? (long long)__ldg(g.rev + k)
                                       : lower_bound_col(g.col, __ldg(g.off + w), __ldg(g.off + w + 1), v);
        return __ldcg(g.cf + ra);
    }
    if (!in) {  // out slot of v: arc v -> w; its reverse residual is its flow
        w = __ldg(g.col + k);
        return DIR == kBfsBackward ? __ldcg(g.cf + k) : __ldcg(g.bf + k);
    }
    w = __ldg(g.in_col + k);  // in slot of v: arc w -> v, out slot j
    const unsigned j = __ldg(g.flow_idx + k);
    return DIR == kBfsBackward ? __ldcg(g.bf + j) : __ldcg(g.cf + j);
}

// The level array of a BFS direction: heights (backward) or cut marks.
template <int DIR>
__device__ __forceinline__ int *bfs_levels(const Params &P)
{
    return DIR == kBfsBackward ? P.st.h : P.st.count;
}
template <int DIR>
__device__ __forceinline__ int bfs_unvisited()
{
    return DIR == kBfsBackward ? kUnvisited : 0;
}

template <int L, int DIR>
__device__ __forceinline__ void bu_found(Ctx &c, int v, long long deg, int val, int nset, int n3)
{
    __stcg(bfs_levels<DIR>(c.P) + v, val);
    c.fe += deg;
    const int cls = classify(c.P, deg);
    if (cls == 2) hub_append(c, n3, nset, v, deg, false, 0, kWChunk, hub_lead<L>(c.P.g, v));
    else q_append(c, n3, nset, cls, v);
}


// Scan W-lane groups of NB entries of v's row starting at row index r0 + sl;
// true if one of them is a residual arc into the frontier.
template <int L, int DIR, int W, int NB>
__device__ __forceinline__ bool bu_scan(const Params &P, int v, long long ob, long long dout, long long ib,
                                        long long deg, long long r0, int sl, int want)
{
    int w[NB], r[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        const long long rr = r0 + sl + (long long)q * W;
        r[q] = 0;
        w[q] = 0;
        if (rr < deg) {
            bool in;
            const long long k = row_slot<L>(ob, dout, ib, rr, in);
            r[q] = bu_res<L, DIR>(P, v, k, in, w[q]);
        }
    }
    const int *lvl = bfs_levels<DIR>(P);
    bool hit = false;
#pragma unroll
    for (int q = 0; q < NB; ++q) hit |= r[q] > 0 && __ldcg(lvl + w[q]) == want;
    return hit;
}

template <int L, int DIR>
__device__ void bfs_level_bu(Ctx &c, int val)
{
    const Params &P = c.P;
    const GraphDev &g = P.g;
    const int gen = c.gen, n3 = (gen + 1) % 3, nset = (gen + 1) & 1;
    const int want = val - 1;
    const long long n = g.n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    reset_rotating(c, gen);
    long long scanned = 0;
    const long long span = (long long)kBlock * kBuVerts;
    if (threadIdx.x == 0) {
        c.sm.ndfr_lo = 0;
        c.sm.ndfr_hi = 0;
    }
    __syncthreads();
    for (long long base = (long long)c.bid * span; base < n; base += (long long)c.nblk * span) {
        int v[kBuVerts];
        long long ob[kBuVerts], dout[kBuVerts], ib[kBuVerts], deg[kBuVerts];
        bool live[kBuVerts];
#pragma unroll
        for (int i = 0; i < kBuVerts; ++i) {
            v[i] = (int)(base + (long long)i * kBlock + threadIdx.x);
            live[i] = v[i] < n && __ldcg(bfs_levels<DIR>(P) + v[i]) == bfs_unvisited<DIR>();
        }
#pragma unroll
        for (int i = 0; i < kBuVerts; ++i) {
            ob[i] = dout[i] = ib[i] = deg[i] = 0;
            if (live[i]) {
                ob[i] = __ldg(g.off + v[i]);
                dout[i] = __ldg(g.off + v[i] + 1) - ob[i];
                deg[i] = dout[i];
                if (L == kRCSR) {
                    ib[i] = __ldg(g.in_off + v[i]);
                    deg[i] += __ldg(g.in_off + v[i] + 1) - ib[i];
                }
                if (deg[i] == 0) {
                    live[i] = false;
                } else if (deg[i] > kBuThread) {
                    live[i] = false;
                    if (classify(P, deg[i]) == 2) c.sm.dfr[span - 1 - atomicAdd(&c.sm.ndfr_hi, 1u)] = v[i];
                    else c.sm.dfr[atomicAdd(&c.sm.ndfr_lo, 1u)] = v[i];
                }
            }
        }
        for (long long r0 = 0; r0 < kBuThread; r0 += kBuStep) {
            bool any = false;
#pragma unroll
            for (int i = 0; i < kBuVerts; ++i) any |= live[i];
            if (!any) break;
            bool hit[kBuVerts];
#pragma unroll
            for (int i = 0; i < kBuVerts; ++i) {
                hit[i] = false;
                if (live[i]) hit[i] = bu_scan<L, DIR, 1, kBuStep>(P, v[i], ob[i], dout[i], ib[i], deg[i], r0, 0, want);
            }
#pragma unroll
            for (int i = 0; i < kBuVerts; ++i) {
                if (!live[i]) continue;
                const long long left = deg[i] - r0;
                scanned += left < kBuStep ? left : kBuStep;
                if (hit[i]) bu_found<L, DIR>(c, v[i], deg[i], val, nset, n3);
                if (hit[i] || left <= kBuStep) live[i] = false;
            }
        }
        __syncthreads();
        // Rows longer than kBuThread: one warp each.  Hub rows too, for their
        // first kBuHubHead entries: the scan usually stops there (rows are
        // sorted by neighbour id, and a renumbered graph puts the largest
        // vertices, the likeliest parents, first), and a renumbered graph
        // also puts whole runs of hubs into one block's vertex range, which
        // one hub at a time on the whole block would take in turn.
        const unsigned nlo = c.sm.ndfr_lo, nhi = c.sm.ndfr_hi;
        for (unsigned i = warp; i < nlo + nhi; i += kWarps) {
            const bool hub = i >= nlo;
            int *slot = hub ? &c.sm.dfr[span - 1 - (i - nlo)] : &c.sm.dfr[i];
            const int u = *slot;
            const long long o = __ldg(g.off + u), dO = __ldg(g.off + u + 1) - o;
            long long ii = 0, d = dO;
            if (L == kRCSR) {
                ii = __ldg(g.in_off + u);
                d += __ldg(g.in_off + u + 1) - ii;
            }
            const long long lim = hub && d > kBuHubHead ? kBuHubHead : d;
            bool found = false;
            for (long long r0 = 0; r0 < lim; r0 += 32 * kBuStep) {
                const bool h1 = bu_scan<L, DIR, 32, kBuStep>(P, u, o, dO, ii, lim, r0, lane, want);
                if (lane == 0) scanned += lim - r0 < 32 * kBuStep ? lim - r0 : 32 * kBuStep;
                if (__any_sync(kFull, h1)) {
                    if (lane == 0) bu_found<L, DIR>(c, u, d, val, nset, n3);
                    found = true;
                    break;
                }
            }
            if (hub && lane == 0 && (found || lim == d)) *slot = -1;  // settled: no block scan
        }
        __syncthreads();
        // the rest of the hub rows not settled by their head: the whole block,
        // kBlock * kBuStep entries per step
        for (unsigned i = 0; i < nhi; ++i) {
            const int u = c.sm.dfr[span - 1 - i];
            if (u < 0) continue;  // block-uniform: read after the barrier above
            const long long o = __ldg(g.off + u), dO = __ldg(g.off + u + 1) - o;
            long long ii = 0, d = dO;
            if (L == kRCSR) {
                ii = __ldg(g.in_off + u);
                d += __ldg(g.in_off + u + 1) - ii;
            }
            for (long long r0 = kBuHubHead; r0 < d; r0 += (long long)kBlock * kBuStep) {
                const bool h1 = bu_scan<L, DIR, kBlock, kBuStep>(P, u, o, dO, ii, d, r0, threadIdx.x, want);
                if (threadIdx.x == 0) scanned += d - r0 < kBlock * kBuStep ? d - r0 : kBlock * kBuStep;
                if (__syncthreads_or(h1)) {
                    if (threadIdx.x == 0) bu_found<L, DIR>(c, u, d, val, nset, n3);
                    break;
                }
            }
        }
        __syncthreads();
        const bool flush = c.sm.qcnt[0] > (unsigned)(kQueueCap / 2) || c.sm.qcnt[1] > (unsigned)(kQueueCap / 2);
        __syncthreads();
        if (threadIdx.x == 0) {
            c.sm.ndfr_lo = 0;
            c.sm.ndfr_hi = 0;
        }
        if (flush) q_flush(c, n3, nset);  // block-uniform; starts with a barrier
        __syncthreads();
    }
    q_flush(c, n3, nset);
    if (scanned) atomicAdd((unsigned long long *)&c.sm.stats[kStatGrArcs], (u64)scanned);
    const long long bfe = block_sum(c, c.fe);   // the next frontier's entries, for the direction rule
    if (threadIdx.x == 0 && bfe) atomicAdd((u64 *)&P.st.ctl->fedges[n3], (u64)bfe);
    c.fe = 0;
}

// Capacity of the out-arcs from the marked side (mark != 0) to the rest,
// initial capacities; this thread's share (valid once it returns true).
// Rows of up to kBuThread entries are summed by one thread (kBuVerts vertices
// at once).  Longer rows are queued in the next (empty) queue generation and,
// after a barrier, taken across the grid: a warp per row, hub rows in
// kWChunk-entry chunks taken by warps.  R-MAT places its long rows at low
// ids, so rows handled by the block that found them would all land on a few
// blocks.
template <int L>
__device__ bool cut_capacity(Ctx &c, long long &sum)
{
    const Params &P = c.P;
    const GraphDev &g = P.g;
    const int *mark = P.st.count;
    const long long n = g.n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long span = (long long)kBlock * kBuVerts;
    const int n3 = (c.gen + 1) % 3, nset = (c.gen + 1) & 1;  // generation c.gen + 1 is empty
    sum = 0;
    for (long long base = (long long)c.bid * span; base < n; base += (long long)c.nblk * span) {
        long long ob[kBuVerts], deg[kBuVerts];
        bool live[kBuVerts];
#pragma unroll
        for (int i = 0; i < kBuVerts; ++i) {
            const long long v = base + (long long)i * kBlock + threadIdx.x;
            live[i] = v < n && __ldcg(mark + v) != 0;
        }
#pragma unroll
        for (int i = 0; i < kBuVerts; ++i) {
            ob[i] = deg[i] = 0;
            if (live[i]) {
                const long long v = base + (long long)i * kBlock + threadIdx.x;
                ob[i] = __ldg(g.off + v);
                deg[i] = __ldg(g.off + v + 1) - ob[i];
                if (deg[i] > kBuThread) {
                    live[i] = false;
                    if (classify(P, deg[i]) == 2)
                        hub_append(c, n3, nset, (int)v, deg[i], false, 0, kWChunk, hub_lead<L>(g, (int)v));
                    else q_append(c, n3, nset, 1, (int)v);
                }
            }
        }
        for (long long r0 = 0; r0 < kBuThread; r0 += kBuStep) {
            bool any = false;
#pragma unroll
            for (int i = 0; i < kBuVerts; ++i) any |= live[i] && r0 < deg[i];
            if (!any) break;
            int w[kBuVerts][kBuStep], cap[kBuVerts][kBuStep];
#pragma unroll
            for (int i = 0; i < kBuVerts; ++i)
#pragma unroll
                for (int q = 0; q < kBuStep; ++q) {
                    const bool ok = live[i] && r0 + q < deg[i];
                    w[i][q] = ok ? __ldg(g.col + ob[i] + r0 + q) : 0;
                    cap[i][q] = ok ? __ldg(g.cf0 + ob[i] + r0 + q) : 0;
                }
#pragma unroll
            for (int i = 0; i < kBuVerts; ++i)
#pragma unroll
                for (int q = 0; q < kBuStep; ++q)
                    if (cap[i][q] && !__ldcg(mark + w[i][q])) sum += cap[i][q];
        }
    }
    q_flush(c, n3, nset);
    if (!grid_sync(c, 33)) return false;
    // rows longer than kBuThread: one warp each, taken across the grid
    {
        const unsigned nmed = __ldcg(&P.st.ctl->q_count[n3][1]);
        const int *q1 = P.st.q[nset][1];
        for (unsigned i = (unsigned)(c.bid * kWarps + warp); i < nmed; i += c.nblk * kWarps) {
            const int u = __ldcg(q1 + i);
            const long long b = __ldg(g.off + u), e = __ldg(g.off + u + 1);
            for (long long k0 = b; k0 < e; k0 += 32 * kBuStep) {
                int w[kBuStep], cap[kBuStep];
#pragma unroll
                for (int q = 0; q < kBuStep; ++q) {
                    const long long k = k0 + q * 32 + lane;
                    w[q] = k < e ? __ldg(g.col + k) : 0;
                    cap[q] = k < e ? __ldg(g.cf0 + k) : 0;
                }
#pragma unroll
                for (int q = 0; q < kBuStep; ++q)
                    if (cap[q] && !__ldcg(mark + w[q])) sum += cap[q];
            }
        }
    }

    // hub rows: chunks of kWChunk entries (starting on a 16-byte boundary in
    // BCSR, as in a push-relabel pass) taken by warps, the hub's row bounds
    // kept across a warp's consecutive chunks
    const u64 hp = __ldcg(&P.st.ctl->hub_pack[n3]);
    const unsigned nh = (unsigned)(hp >> 40), nchunks = (unsigned)(hp & kChunkMask);
    unsigned pos, j, nch;
    if (nchunks) {
        WGrab gb(nchunks, c.nblk * kWarps);
        while (grab_wchunk<L>(c, n3, nset, nh, nchunks, gb, pos, j, nch)) {
            const long long lo = (long long)j * kWChunk - (L == kBCSR ? (gb.ob & 3) : 0);
            constexpr int NB = kWChunk / 32;
            int w[NB], cap[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const long long r = lo + lane + 32LL * q;
                const bool ok = r >= 0 && r < gb.dout;
                w[q] = ok ? __ldg(g.col + gb.ob + r) : 0;
                cap[q] = ok ? __ldg(g.cf0 + gb.ob + r) : 0;
            }
#pragma unroll
            for (int q = 0; q < NB; ++q)
                if (cap[q] && !__ldcg(mark + w[q])) sum += cap[q];
        }
    }
    return true;
}

// Direction of the next BFS level (after Beamer, Asanovic and Patterson):
// bottom-up when the frontier holds at least bottom_up_min vertices and,
// by the entry rule, its residual-list entries times bottom_up reach the
// entries of the vertices not yet visited (nor written off); by the vertex
// rule, its vertex count times bottom_up must reach the unvisited vertices.
// bottom_up_edges: 0 = vertex rule, 1 = entry rule, 2 = entry rule where
// `entry_ok` (the searches of phase 1 and of the cut), vertex rule in the
// searches of phase 2, where many unvisited vertices never find a parent and
// a bottom-up level scans their whole rows.
__device__ __forceinline__ bool bottom_up_level(const Params &P, unsigned tot, long long fe, long long unseen_edges,
                                                long long unseen, bool entry_ok)
{
    if (P.bottom_up <= 0 || tot < (unsigned)P.bottom_up_min) return false;
    if (P.bottom_up_edges == 1 || (P.bottom_up_edges == 2 && entry_ok)) return fe * P.bottom_up >= unseen_edges;
    return (long long)tot * P.bottom_up >= unseen;
}

// Seed a BFS: generation `gen` holds the single vertex v.
template <int L>
__device__ __forceinline__ void seed_queue(Ctx &c, int gen, int v)
{
    if (c.bid == 0 && threadIdx.x == 0) {
        const long long d = degree<L>(c.P.g, v);
        const int cls = classify(c.P, d);
        c.P.st.q[gen & 1][cls][0] = v;
        c.P.st.ctl->fedges[gen % 3] = d;
        if (cls == 2) {
            const unsigned nch = hub_chunks(d, kWChunk, hub_lead<L>(c.P.g, v));
            c.P.st.hub_start[gen & 1][0] = 0;
            for (unsigned j = 0; j < nch; ++j) c.P.st.hub_chunk[gen & 1][j] = 0;
            c.P.st.ctl->hub_pack[gen % 3] = (1ull << 40) | nch;
        } else {
            c.P.st.ctl->q_count[gen % 3][cls] = 1;
        }
    }
}

// Global relabel (§2.2): heights = base + BFS distance to `target` over
// residual arcs, never through `excluded`; unreachable vertices get
// `unreach` and a mark in dead[] that later global relabels of the phase
// skip.  Phase 1 writes off the excess of newly unreachable vertices
// (Excess_total -= e(v), once per vertex) and rebuilds the gap counts; in
// phase 2 an unreachable vertex holds no excess (all excess can return to s).
template <int L, int SW>
__device__ bool global_relabel(Ctx &c, bool phase1, bool first_of_phase2 = false)
{
    const Params &P = c.P;
    const GraphDev &g = P.g;
    const int n = g.n;
    const int target = phase1 ? g.t : g.s;
    const int excluded = phase1 ? g.s : g.t;
    const int base = phase1 ? 0 : n;
    const int unreach = phase1 ? n : 2 * n;
    const bool gap = phase1 && P.gap;
    if (c.bid == 0 && threadIdx.x == 0) {
        c.gr_start_ns = global_ns();
        if (first_of_phase2) {  // the marks are cleared below
            P.st.ctl->dead_count = 0;
            P.st.ctl->dead_edges = 0;
        }
    }
    const long long stride = (long long)c.nblk * kBlock;
    // Four vertices per thread and step (16-byte height and count stores,
    // 4-byte reads of the marks), the last n mod 4 and count[n] one by one.
    const long long n4 = (long long)n & ~3LL;
    for (long long q = c.bid * kBlock + threadIdx.x; 4 * q < n4; q += stride) {
        const long long v0 = 4 * q;
        if (gap) __stcg(reinterpret_cast<int4 *>(P.st.count) + q, make_int4(0, 0, 0, 0));
        uchar4 d4 = make_uchar4(0, 0, 0, 0);
        if (first_of_phase2) reinterpret_cast<uchar4 *>(P.st.dead)[q] = d4;  // phase 1's marks mean "cannot reach t"
        else d4 = reinterpret_cast<const uchar4 *>(P.st.dead)[q];
        const unsigned char d[4] = {d4.x, d4.y, d4.z, d4.w};
        bool all = true;
#pragma unroll
        for (int i = 0; i < 4; ++i) all = all && !d[i] && v0 + i != excluded;
        if (all) {
            int4 hv = make_int4(kUnvisited, kUnvisited, kUnvisited, kUnvisited);
            if (target >= v0 && target < v0 + 4) (&hv.x)[target - v0] = base;
            __stcg(reinterpret_cast<int4 *>(P.st.h) + q, hv);
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (!d[i] && v0 + i != excluded) __stcg(P.st.h + v0 + i, v0 + i == target ? base : kUnvisited);
        }
    }
    for (long long v = n4 + c.bid * kBlock + threadIdx.x; v <= n; v += stride) {
        if (gap) __stcg(P.st.count + v, 0);
        if (v == n || v == excluded) continue;
        if (first_of_phase2) P.st.dead[v] = 0;
        else if (P.st.dead[v]) continue;
        __stcg(P.st.h + v, v == target ? base : kUnvisited);
    }
    seed_queue<L>(c, c.gen, target);
    if (!grid_sync(c, 10)) return false;
    // Direction choice (after Beamer et al.): a level runs bottom-up when its
    // frontier, times bottom_up, reaches the vertices not yet visited (those
    // neither reached nor marked unreachable by an earlier global relabel)
    // and holds at least bottom_up_min vertices.  Uniform over the team: every
    // block reads the same counters after the barrier.  Vertices that cannot reach the target
    // are marked (dead[]) and skipped by the later global relabels of the
    // phase, so bottom-up levels do not rescan their rows: no residual path
    // to the target can appear for them, because no push ever enters a
    // vertex at the height cap.
    long long seen = __ldcg(&P.st.ctl->dead_count);
    long long unseen_edges = (L == kRCSR ? 2 : 1) * g.slots - __ldcg(&P.st.ctl->dead_edges);
    for (int level = 0;; ++level) {
        const unsigned tot = queue_total(P.st.ctl, c.gen);
        if (tot == 0) break;
        if (gap && c.bid == 0 && threadIdx.x == 0 && level < n) __stcg(P.st.count + level, (int)tot);
        seen += tot;
        const long long fe = __ldcg(&P.st.ctl->fedges[c.gen % 3]);
        unseen_edges -= fe;
        const bool bu_mode = bottom_up_level(P, tot, fe, unseen_edges, (long long)n - seen, phase1);
        if (bu_mode)
            bfs_level_bu<L, kBfsBackward>(c, base + level + 1);
        else
            bfs_level<L, kBfsBackward, SW>(c, base + level + 1);
        if (!grid_sync(c, bu_mode ? 13 : 11)) return false;  // trace id: bottom-up or top-down level
        c.gen++;
    }
    long long wo = 0, nd = 0, nde = 0;
    // Unreached vertices: the height cap, a mark, and (phase 1) the write-off.
    // Four heights per thread and step (one 16-byte read), the last n mod 4
    // one by one.
    auto finish = [&](long long v) {
        __stcg(P.st.h + v, unreach);
        if (!P.st.dead[v]) {
            P.st.dead[v] = 1;
            ++nd;
            nde += degree<L>(g, (int)v);
            if (phase1) wo += __ldcg(P.st.e + v);
        }
    };
    for (long long q = c.bid * kBlock + threadIdx.x; 4 * q < n4; q += stride) {
        const int4 hv = __ldcg(reinterpret_cast<const int4 *>(P.st.h) + q);
        const int h4[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (h4[i] == kUnvisited && 4 * q + i != excluded) finish(4 * q + i);
    }
    for (long long v = n4 + c.bid * kBlock + threadIdx.x; v < n; v += stride)
        if (v != excluded && __ldcg(P.st.h + v) == kUnvisited) finish(v);
    long long bw = block_sum(c, wo);
    if (threadIdx.x == 0 && bw) {
        atomicAdd((u64 *)&P.st.ctl->excess_total, (u64)(-bw));
        atomicAdd((u64 *)&P.st.ctl->written_off, (u64)bw);
    }
    const long long bd = block_sum(c, nd);
    if (threadIdx.x == 0 && bd) atomicAdd((u64 *)&P.st.ctl->dead_count, (u64)bd);
    const long long bde = block_sum(c, nde);
    if (threadIdx.x == 0 && bde) atomicAdd((u64 *)&P.st.ctl->dead_edges, (u64)bde);
    if (c.bid == 0 && threadIdx.x == 0) P.st.ctl->global_relabels++;
    const bool ok = grid_sync(c, 12);
    if (c.bid == 0 && threadIdx.x == 0) {
        c.gr_end_ns = global_ns();
        c.gr_ns = c.gr_end_ns - c.gr_start_ns;
    }
    return ok;
}

// `max_it` iterations of Alg. 2 (fewer if the AVQ empties).  Returns false
// on a device error; *it_done receives the count.
template <int L, int SW>
__device__ bool iterate(Ctx &c, bool phase1, long long max_it, long long *it_total)
{
    const Params &P = c.P;
    const int hcap = phase1 ? P.g.n : 2 * P.g.n;
    // avq_incremental = 2: after a pass whose AVQ held at most 64 vertices
    // per block and no hub (or a block-local pass that processed that few
    // and deferred nothing), the next pass runs block-locally (pr_local).
    const unsigned local_max = 64u * c.nblk;
    bool local = false;
    for (long long i = 0; i < max_it; ++i) {
        // Time-balanced global relabel: once the iterations since the last
        // global relabel have taken gr_ratio times as long as it did.
        // The flag names the generation whose iteration raised it, so it never
        // needs clearing (a clear could race with a slower block's read).
        if (i > 0 && P.gr_ratio > 0.f && __ldcg(&P.st.ctl->gr_due_gen) == c.gen - 1) break;
        if (P.thread_centric) {
            tc_process<L>(c, phase1, hcap);
            if (c.bid == 0 && threadIdx.x == 0 && P.gr_ratio > 0.f) {
                const u64 now = global_ns();
                if ((float)(now - c.gr_end_ns) >= P.gr_ratio * (float)c.gr_ns) P.st.ctl->gr_due_gen = c.gen;
            }
            if (!grid_sync(c, 22)) return false;
            const bool none = __ldcg(&P.st.ctl->q_count[c.gen % 3][0]) == 0;
            reset_rotating(c, c.gen);  // every block has read generation gen - 1's gap candidate
            c.gen++;
            if (none) break;  // no active vertex was found: nothing was pushed
            ++*it_total;
            if (*it_total >= P.max_iterations) {
                if (c.bid == 0 && threadIdx.x == 0) {
                    atomicCAS(&P.st.ctl->err, 0, (int)WBPR_ETIMEOUT);
                    P.st.ctl->err_where = 23;
                }
                return false;
            }
            continue;
        }
        if (local && phase1 && P.gap) {  // a pending gap needs a full compaction
            const int cand = __ldcg(&P.st.ctl->gap_level[(c.gen + 2) % 3]);
            if (cand < P.g.n && __ldcg(P.st.count + cand) == 0) local = false;
        }
        if (local) {
            pr_local<L, SW>(c, phase1, hcap);
            if (c.bid == 0 && threadIdx.x == 0 && P.gr_ratio > 0.f) {
                const u64 now = global_ns();
                if ((float)(now - c.gr_end_ns) >= P.gr_ratio * (float)c.gr_ns) P.st.ctl->gr_due_gen = c.gen;
            }
            if (!grid_sync(c, 24)) return false;
            const unsigned na = __ldcg(&P.st.ctl->local_active[c.gen % 3]);
            const bool deferred = __ldcg(&P.st.ctl->local_defer[c.gen % 3]) != 0;
            reset_rotating(c, c.gen);  // every block has read generation gen - 1's gap candidate
            c.gen++;
            if (na == 0 && !deferred) break;  // no vertex was active: as an empty AVQ
            local = !deferred && na <= local_max;
        } else {
            build_avq<L>(c, phase1, hcap, i == 0);
            if (!grid_sync(c, 20)) return false;
            const unsigned tot = queue_total(P.st.ctl, c.gen);
            const bool hubs = (__ldcg(&P.st.ctl->hub_pack[c.gen % 3]) >> 40) != 0;
            if (tot == 0) {
                reset_rotating(c, c.gen);
                if (!grid_sync(c, 21)) return false;
                c.gen++;
                break;
            }
            pr_process<L, SW>(c, phase1, hcap);
            if (c.bid == 0 && threadIdx.x == 0 && P.gr_ratio > 0.f) {
                const u64 now = global_ns();
                if ((float)(now - c.gr_end_ns) >= P.gr_ratio * (float)c.gr_ns) P.st.ctl->gr_due_gen = c.gen;
            }
            if (!grid_sync(c, 22)) return false;
            c.gen++;
            local = P.local_passes && P.st.touch && !hubs && tot <= local_max;
        }
        ++*it_total;
        if (*it_total >= P.max_iterations) {
            if (c.bid == 0 && threadIdx.x == 0) {
                atomicCAS(&P.st.ctl->err, 0, (int)WBPR_ETIMEOUT);
                P.st.ctl->err_where = 23;
            }
            return false;
        }
    }
    return true;
}

template <int L, int SW>
__device__ bool run_phase(Ctx &c, bool phase1, long long *it_total)
{
    const Params &P = c.P;
    Ctl *ctl = P.st.ctl;
    if (!global_relabel<L, SW>(c, phase1, !phase1)) return false;
    int idle_rounds = 0;
    for (;;) {
        const long long es = __ldcg(P.st.e + P.g.s), et = __ldcg(P.st.e + P.g.t);
        const long long goal = phase1 ? __ldcg(&ctl->excess_total) : __ldcg(&ctl->preflow_total);
        if (es + et >= goal) break;
        const long long before = *it_total;
        if (!iterate<L, SW>(c, phase1, P.cycle, it_total)) return false;
        // A global relabel right after an empty AVQ must settle the test above;
        // two rounds in a row without any iteration mean it cannot: give up
        // instead of looping.
        idle_rounds = (*it_total == before) ? idle_rounds + 1 : 0;
        if (idle_rounds >= 2) {
            if (c.bid == 0 && threadIdx.x == 0) {
                atomicCAS(&ctl->err, 0, (int)WBPR_ESTATE);
                ctl->err_where = 24;
            }
            return false;
        }
        if (!global_relabel<L, SW>(c, phase1)) return false;
    }
    return true;
}

// Reset the residual graph and state, then the preflow of Alg. 1 step 0.
// The mirror cfb[a] = cf[rev[a]] is reset to cf0[rev[a]] without a gather: a
// push moves capacity between the two slots of a pair, so cf[a] + cf[rev[a]]
// (= cf[a] + cfb[a]) stays cf0[a] + cf0[rev[a]] in every state the solver
// leaves behind (the builder starts from cf = cf0, cfb = cf0[rev]).  Only a
// caller whose arrays may hold another graph's state asks for the gather.
template <int L>
__device__ bool preflow(Ctx &c)
{
    const Params &P = c.P;
    const GraphDev &g = P.g;
    const long long stride = (long long)c.nblk * kBlock;
    const long long tid = c.bid * kBlock + threadIdx.x;
    // Four slots per thread and step with 16-byte accesses when every array
    // is 16-byte aligned (more bytes in flight per thread); the rest, and the
    // gather, one slot at a time.
    const bool mirror = L == kBCSR && g.cfb;
    const bool vec = !(mirror && P.mirror_gather) &&
                     ((reinterpret_cast<uintptr_t>(g.cf0) | reinterpret_cast<uintptr_t>(g.cf) |
                       reinterpret_cast<uintptr_t>(mirror ? g.cfb : g.cf) |
                       reinterpret_cast<uintptr_t>(L == kRCSR ? g.bf : g.cf)) & 15) == 0;
    const long long first = vec ? (g.slots & ~3LL) : 0;
    if (vec) {
        const int4 *cf0v = reinterpret_cast<const int4 *>(g.cf0);
        int4 *cfv = reinterpret_cast<int4 *>(g.cf);
        for (long long q = tid; q < (first >> 2); q += stride) {
            const int4 c0 = __ldg(cf0v + q);
            if (mirror) {
                int4 *cfbv = reinterpret_cast<int4 *>(g.cfb);
                const int4 f = __ldcg(cfv + q);
                int4 b = __ldcg(cfbv + q);
                b.x += f.x - c0.x;
                b.y += f.y - c0.y;
                b.z += f.z - c0.z;
                b.w += f.w - c0.w;
                __stcg(cfbv + q, b);
            }
            __stcg(cfv + q, c0);
            if (L == kRCSR) __stcg(reinterpret_cast<int4 *>(g.bf) + q, make_int4(0, 0, 0, 0));
        }
    }
    for (long long k = first + tid; k < g.slots; k += stride) {
        const int c0 = __ldg(g.cf0 + k);
        if (mirror) {
            if (P.mirror_gather) g.cfb[k] = __ldg(g.cf0 + __ldg(g.rev + k));
            else g.cfb[k] = __ldcg(g.cf + k) + __ldcg(g.cfb + k) - c0;
        }
        g.cf[k] = c0;
        if (L == kRCSR) g.bf[k] = 0;
    }
    for (long long v = tid; v < g.n; v += stride) {
        P.st.e[v] = 0;
        P.st.h[v] = (v == g.s) ? g.n : 0;
        P.st.dead[v] = 0;
    }
    if (!grid_sync(c, 1)) return false;
    const long long b = __ldg(g.off + g.s), e = __ldg(g.off + g.s + 1);
    long long sum = 0;
    for (long long k = b + tid; k < e; k += stride) {
        int cap = g.cf[k];
        if (cap <= 0) continue;
        g.cf[k] = 0;
        int v = __ldg(g.col + k);
        if (L == kBCSR) {
            long long ra = P.use_rev ? (long long)__ldg(g.rev + k)
                                     : lower_bound_col(g.col, __ldg(g.off + v), __ldg(g.off + v + 1), g.s);
            atomicAdd(g.cf + ra, cap);
            if (g.cfb) {
                atomicAdd(g.cfb + k, cap);
                atomicSub(g.cfb + ra, cap);
            }
        } else {
            atomicAdd(g.bf + k, cap);
        }
        atomicAdd((u64 *)(P.st.e + v), (u64)cap);
        sum += cap;
    }
    long long bs = block_sum(c, sum);
    if (threadIdx.x == 0 && bs) {
        atomicAdd((u64 *)&P.st.ctl->excess_total, (u64)bs);
        atomicAdd((u64 *)&P.st.ctl->preflow_total, (u64)bs);
    }
    return grid_sync(c, 2);
}

// Forward BFS from s over residual arcs; source_side and cut capacity.
template <int L, int SW>
__device__ bool min_cut(Ctx &c)
{
    const Params &P = c.P;
    const GraphDev &g = P.g;
    const int n = g.n;
    const long long stride = (long long)c.nblk * kBlock;
    const long long tid = c.bid * kBlock + threadIdx.x;
    int *mark = P.st.count;  // 0 = not reached, else BFS level + 1
    for (long long v = tid; v <= n; v += stride) __stcg(mark + v, v == g.s ? 1 : 0);
    seed_queue<L>(c, c.gen, g.s);
    if (!grid_sync(c, 30)) return false;
    // Forward BFS from s, bottom-up on large frontiers (the forward residual
    // w -> v of an entry of v's row: the mirror cfb in BCSR, else a lookup of
    // the reverse slot).
    long long seen = 0;
    long long unseen_edges = (L == kRCSR ? 2 : 1) * g.slots;
    for (int level = 0;; ++level) {
        const unsigned tot = queue_total(P.st.ctl, c.gen);
        if (tot == 0) break;
        seen += tot;
        const long long fe = __ldcg(&P.st.ctl->fedges[c.gen % 3]);
        unseen_edges -= fe;
        const bool bu_mode = bottom_up_level(P, tot, fe, unseen_edges, (long long)n - seen, true);
        if (bu_mode)
            bfs_level_bu<L, kBfsForward>(c, level + 2);
        else
            bfs_level<L, kBfsForward, SW>(c, level + 2);
        if (!grid_sync(c, bu_mode ? 34 : 31)) return false;  // trace id: bottom-up or top-down level
        c.gen++;
    }
    long long sum = 0;
    if (!cut_capacity<L>(c, sum)) return false;
    long long bs = block_sum(c, sum);
    if (threadIdx.x == 0 && bs) atomicAdd((u64 *)&P.st.ctl->cut_value, (u64)bs);
    // the cut side in input ids: a renumbered handle gathers through the
    // inverse order, so that the byte writes stay coalesced
    if (P.source_side)
        for (long long i = tid; i < n; i += stride)
            P.source_side[i] = (unsigned char)(__ldcg(mark + (g.perm ? __ldg(g.perm + i) : i)) != 0);
    return grid_sync(c, 32);
}

// At least WBPR_MIN_BLOCKS resident blocks per SM: the solver is bound by
// memory latency, so occupancy (more warps in flight) matters more than the
// few registers it costs.
#ifndef WBPR_MIN_BLOCKS
#define WBPR_MIN_BLOCKS 4
#endif

// One whole solve (the modes in P.mode) by the calling team of blocks.
template <int L, int SW>
__device__ __forceinline__ void solve_instance(Ctx &c)
{
    const Params &P = c.P;
    Smem &sm = c.sm;
    if (threadIdx.x < kClasses) sm.qcnt[threadIdx.x] = 0;
    if (threadIdx.x < kStatCount) sm.stats[threadIdx.x] = 0;
    if (c.bid == 0 && threadIdx.x == 0) {
        for (int k = 0; k < 3; ++k) P.st.ctl->gap_level[k] = kUnvisited;
        P.st.ctl->gr_due_gen = -1;
    }
    __syncthreads();
    long long it_total = 0;
    bool ok = true;
    if (P.mode & kModePreflow) ok = preflow<L>(c);
    if (ok && (P.mode & kModePhase1)) {
        ok = run_phase<L, SW>(c, true, &it_total);
        if (c.bid == 0 && threadIdx.x == 0) P.st.ctl->phase1_iterations = it_total;
    }
    if (ok && (P.mode & kModeGrOnce)) ok = global_relabel<L, SW>(c, true);
    if (ok && (P.mode & kModeIters)) ok = iterate<L, SW>(c, true, P.iters_arg, &it_total);
    if (ok && (P.mode & kModePhase2)) ok = run_phase<L, SW>(c, false, &it_total);
    if (ok && (P.mode & kModeCut)) ok = min_cut<L, SW>(c);
    if (c.bid == 0 && threadIdx.x == 0) P.st.ctl->iterations = it_total;
    __syncthreads();
    if (threadIdx.x < kStatCount) P.st.bstats[(long long)c.bid * kStatCount + threadIdx.x] = sm.stats[threadIdx.x];
    __syncthreads();
}

template <int L, int SW>
__global__ void __launch_bounds__(kBlock, WBPR_MIN_BLOCKS) solve_kernel(Params P)
{
    __shared__ Smem sm;
    extern __shared__ __align__(16) int dyn_smem[];
    Ctx c{P, sm, 0ull, 0, gridDim.x, blockIdx.x, 0ull, 0ull, 0ull,
          dynamic_smem_bytes() >= (unsigned)kStageBytes ? dyn_smem : nullptr, 0};
    solve_instance<L, SW>(c);
}

// Barrier over a team of `tsize` blocks (counter `bar`); a single-block team
// is just __syncthreads.  Gives up after `limit_ns`.
__device__ bool team_sync(u64 *bar, unsigned tsize, u64 limit_ns, u64 &target, Smem &sm)
{
    __syncthreads();
    if (tsize > 1 && threadIdx.x == 0) {
        target += tsize;
        __threadfence();
        atomicAdd(bar, 1ULL);
        u64 t0 = 0;
        unsigned spins = 0;
        int ok = 1;
        while (ld_acquire(bar) < target) {
            ++spins;
            if ((spins & 255u) == 0) {
                const u64 now = global_ns();
                if (t0 == 0) t0 = now;
                else if (now - t0 > limit_ns) {
                    ok = 0;
                    break;
                }
            }
            if (spins > 64) __nanosleep(32);
        }
        __threadfence();
        sm.ok = ok;
    } else if (threadIdx.x == 0) {
        sm.ok = 1;
    }
    __syncthreads();
    return sm.ok != 0;
}

__device__ __forceinline__ unsigned ld_acquire_sys_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_sys_s32(int *p, int v)
{
    asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Persistent server: teams wait for requests that the host publishes in
// host-mapped rings (one ring per size class), solve each completely and
// publish the result, until the host raises `stop` or no request has come
// for `idle_ns`.  Blocks [0, n_big_teams * team_big) form teams of team_big
// blocks (class 1, large instances); every other block is a team of one
// (class 0, small instances).
template <int L, int SW>
__global__ void __launch_bounds__(kBlock, WBPR_MIN_BLOCKS) server_kernel(ServerDesc D)
{
    __shared__ Smem sm;
    __shared__ Params sp;
    __shared__ unsigned s_item;
    constexpr unsigned kExit = 0xffffffffu;
    const unsigned nbig = (unsigned)(D.n_big_teams * D.team_big);
    int cls;
    unsigned team, rank, tsize;
    if (blockIdx.x < nbig) {
        cls = 1;
        team = blockIdx.x / D.team_big;
        rank = blockIdx.x % D.team_big;
        tsize = D.team_big;
    } else {
        cls = 0;
        team = D.n_big_teams + (blockIdx.x - nbig);
        rank = 0;
        tsize = 1;
    }
    const u64 team_limit = D.idle_ns + D.timeout_ns;
    u64 target = 0;
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) {
            // Claim the next request only once the host has published it, so a
            // team that leaves (stop flag, idle limit) never strands one.
            unsigned item = kExit;
            const u64 t0 = global_ns();
            unsigned spins = 0;
            for (;;) {
                const unsigned cur = *(volatile unsigned *)(D.next[cls]);
                if (cur >= D.capacity[cls]) {
                    D.team_exit[team] = 1;
                    break;
                }
                if ((u64)cur < ld_acquire((const u64 *)(D.mirror + 2 * cls))) {
                    if (atomicCAS(D.next[cls], cur, cur + 1) == cur) {
                        item = cur;
                        break;
                    }
                    continue;
                }
                // Waiting leaders watch device-memory mirrors of the host's
                // counters; one elected poller at a time refreshes them from the
                // host-mapped words (system-scope loads are costly, and hundreds
                // of leaders issuing them continuously starve other work).
                // The host publishes requests before it raises stop; the poller
                // reads stop first and mirrors the counts before stop, so a
                // leader that sees stop and then re-reads the count sees every
                // request published before it.
                if (ld_acquire((const u64 *)(D.mirror + 4)) != 0) {
                    if ((u64)cur < ld_acquire((const u64 *)(D.mirror + 2 * cls))) continue;
                    D.team_exit[team] = 2;
                    break;
                }
                // The idle limit is checked on every pass, the poller's too: a
                // leader that keeps winning the poll token (the last one waiting)
                // must still leave once no request has come for idle_ns.
                if ((++spins & 63u) == 0 && global_ns() - t0 > D.idle_ns) {
                    D.team_exit[team] = 3;
                    break;
                }
                if (atomicCAS(D.poll_token, 0, 1) == 0) {
                    const unsigned st = ld_acquire_sys_u32((const unsigned *)D.stop);
                    const unsigned a0 = ld_acquire_sys_u32(D.avail[0]);
                    const unsigned a1 = ld_acquire_sys_u32(D.avail[1]);
                    atomicMax((u64 *)(D.mirror + 0), (u64)a0);
                    atomicMax((u64 *)(D.mirror + 2), (u64)a1);
                    __threadfence();
                    if (st) atomicExch((u64 *)(D.mirror + 4), 1ull);
                    __threadfence();
                    atomicExch(D.poll_token, 0);
                    __nanosleep(200);
                    continue;
                }
                __nanosleep(500);
            }
            D.team_item[team] = item;
            s_item = item;
        }
        if (!team_sync(D.team_bar + team, tsize, team_limit, target, sm)) {
            if (threadIdx.x == 0) D.team_exit[team] = 4;
            return;
        }
        if (threadIdx.x == 0 && rank != 0) s_item = __ldcg(D.team_item + team);
        __syncthreads();
        const unsigned item = s_item;
        if (item == kExit) return;
        __threadfence_system();
        const int *src = (const int *)(D.ring[cls] + item);
        for (unsigned i = threadIdx.x; i < sizeof(Params) / sizeof(int); i += kBlock) ((int *)&sp)[i] = src[i];
        __syncthreads();
        const Params &P = sp;
        const u64 t_start = global_ns();
        if (P.g.layout_tag == L) {
            if (rank == 0) {
                for (unsigned i = threadIdx.x; i < sizeof(Ctl) / sizeof(int); i += kBlock) ((int *)P.st.ctl)[i] = 0;
                __threadfence();
            }
            if (!team_sync(D.team_bar + team, tsize, team_limit, target, sm)) {
                if (threadIdx.x == 0) D.team_exit[team] = 5;
                return;
            }
            Ctx c{P, sm, 0ull, 0, tsize, rank, 0ull, 0ull, 0ull, nullptr, 0};
            solve_instance<L, SW>(c);
        }
        if (rank == 0 && threadIdx.x == 0) {
            ServerOut *o = D.out[cls] + item;
            const bool ran = P.g.layout_tag == L;
            o->value = ran ? __ldcg(P.st.e + P.g.t) : -1;
            o->iterations = ran ? __ldcg(&P.st.ctl->iterations) : 0;
            o->err = ran ? __ldcg(&P.st.ctl->err) : (int)WBPR_ESTATE;
            o->t_start = t_start;
            o->t_end = global_ns();
            __threadfence_system();
            st_release_sys_s32(&o->done, 1);
        }
        if (!team_sync(D.team_bar + team, tsize, team_limit, target, sm)) {
            if (threadIdx.x == 0) D.team_exit[team] = 6;
            return;
        }
    }
}

}  // namespace
}  // namespace wbpr
