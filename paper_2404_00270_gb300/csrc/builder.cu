// Graph builder: input arcs (COO, device) -> the residual layouts of §3.2.
//
// BCSR (Fig. 2(d)): every non-loop input arc i = (u,v,c) contributes two
// half-entries, position 2i (row u, col v, capacity c) and position 2i + 1
// (row v, col u, capacity 0).  All half-entries in (row, col) order, ties by
// position, come from three steps: a radix sort of the arcs by (u, v) (the
// tail-side half-entries), a stable sort of that list by v alone (the
// head-side ones, in (v, u) order), and a merge of the two lists.  A merge
// of equal keys then gives one slot per neighbour pair with cf0 = sum of the
// capacities u -> v; rows come out sorted by neighbour id, which the
// binary-search backward lookup of §3.2 needs.  The positions ride along, so
// the two half-entries of an arc land in mutually reverse slots (rev[] and
// arc2slot[] are scatters), and duplicates of (u, v) stay in input order
// inside their run (the edge-flow split's prefix is a scan by key).
// RCSR (Fig. 2(c)): out rows = arcs sorted by (src, dst); in rows = the same
// arcs sorted by (dst, src), each in entry keeping flow_idx, the out slot.
// Keys pack (row, col) into 2 * bitlen(n - 1) bits, so the radix sorts make
// only as many passes as the vertex count needs.  Sorting, merging and scans
// use CUB (device radix sort / merge / scan, header-only).
#include <cub/cub.cuh>
#include <cub/device/device_merge.cuh>
#include <thrust/iterator/counting_iterator.h>
#include <thrust/iterator/transform_iterator.h>
#include <thrust/iterator/transform_output_iterator.h>
#include <thrust/iterator/zip_iterator.h>
#include <thrust/tuple.h>

#include <stdint.h>

#include <string>

#include "handle.h"

namespace wbpr {
namespace {

typedef unsigned long long u64;

// A CUB radix-sort tuning for builds that run while a persistent server
// kernel holds two blocks of every SM (wbpr_options.lean_build): onesweep
// and single-tile blocks of 256 threads with few items per thread, so that
// a sort block fits in the registers and shared memory the server leaves.
// CUB's own tuning for this GPU uses 384-thread onesweep blocks of up to 96
// registers a thread (u64 keys), more than half an SM's register file.
template <typename KeyT, typename ValueT, typename OffsetT>
struct LeanRadixHub {
    using DominantT = ::cuda::std::_If<(sizeof(ValueT) > sizeof(KeyT)), ValueT, KeyT>;
    struct Policy : cub::ChainedPolicy<1000, Policy, Policy> {
        static constexpr bool ONESWEEP = true;
        static constexpr int ONESWEEP_RADIX_BITS = 8;
        using HistogramPolicy = cub::AgentRadixSortHistogramPolicy<128, 8, 1, KeyT, ONESWEEP_RADIX_BITS>;
        using ExclusiveSumPolicy = cub::AgentRadixSortExclusiveSumPolicy<256, ONESWEEP_RADIX_BITS>;
        using OnesweepPolicy =
            cub::AgentRadixSortOnesweepPolicy<256, 12, DominantT, 1, cub::RADIX_RANK_MATCH_EARLY_COUNTS_ANY,
                                              cub::BLOCK_SCAN_RAKING_MEMOIZE, cub::RADIX_SORT_STORE_DIRECT,
                                              ONESWEEP_RADIX_BITS>;
        using ScanPolicy = cub::AgentScanPolicy<256, 8, OffsetT, cub::BLOCK_LOAD_WARP_TRANSPOSE, cub::LOAD_DEFAULT,
                                                cub::BLOCK_STORE_WARP_TRANSPOSE, cub::BLOCK_SCAN_RAKING_MEMOIZE>;
        using DownsweepPolicy =
            cub::AgentRadixSortDownsweepPolicy<256, 8, DominantT, cub::BLOCK_LOAD_TRANSPOSE, cub::LOAD_DEFAULT,
                                               cub::RADIX_RANK_MATCH, cub::BLOCK_SCAN_WARP_SCANS, 6>;
        using AltDownsweepPolicy =
            cub::AgentRadixSortDownsweepPolicy<256, 8, DominantT, cub::BLOCK_LOAD_TRANSPOSE, cub::LOAD_DEFAULT,
                                               cub::RADIX_RANK_MEMOIZE, cub::BLOCK_SCAN_WARP_SCANS, 5>;
        using UpsweepPolicy = cub::AgentRadixSortUpsweepPolicy<256, 8, DominantT, cub::LOAD_DEFAULT, 6>;
        using AltUpsweepPolicy = cub::AgentRadixSortUpsweepPolicy<256, 8, DominantT, cub::LOAD_DEFAULT, 5>;
        using SingleTilePolicy =
            cub::AgentRadixSortDownsweepPolicy<256, 8, DominantT, cub::BLOCK_LOAD_DIRECT, cub::LOAD_LDG,
                                               cub::RADIX_RANK_MEMOIZE, cub::BLOCK_SCAN_WARP_SCANS, 6>;
        using SegmentedPolicy =
            cub::AgentRadixSortDownsweepPolicy<256, 8, DominantT, cub::BLOCK_LOAD_TRANSPOSE, cub::LOAD_DEFAULT,
                                               cub::RADIX_RANK_MEMOIZE, cub::BLOCK_SCAN_WARP_SCANS, 6>;
        using AltSegmentedPolicy =
            cub::AgentRadixSortDownsweepPolicy<256, 8, DominantT, cub::BLOCK_LOAD_TRANSPOSE, cub::LOAD_DEFAULT,
                                               cub::RADIX_RANK_MEMOIZE, cub::BLOCK_SCAN_WARP_SCANS, 5>;
    };
    using MaxPolicy = Policy;
};

// Stable ascending radix sort of key/value pairs over bits [b0, b1), with
// CUB's tuning or, for lean builds, LeanRadixHub's.
template <typename K, typename V>
cudaError_t sort_pairs(bool lean, void *tmp, size_t &bytes, cub::DoubleBuffer<K> &k, cub::DoubleBuffer<V> &v,
                       int64_t n, int b0, int b1, cudaStream_t st)
{
    if (!lean) return cub::DeviceRadixSort::SortPairs(tmp, bytes, k, v, n, b0, b1, st);
    using OffsetT = cub::detail::choose_offset_t<int64_t>;  // the offset type CUB's own entry point picks
    using D = cub::DispatchRadixSort<cub::SortOrder::Ascending, K, V, OffsetT, cub::detail::identity_decomposer_t,
                                     LeanRadixHub<K, V, OffsetT>>;
    return D::Dispatch(tmp, bytes, k, v, (OffsetT)n, b0, b1, true, st);
}

// Arc keys (u << b) | v, self-loops the all-ones key, values the input
// index; ids are checked before use (flag 1: out of range or negative
// capacity).  With perm (a renumbered handle) the key holds the new ids
// perm[u], perm[v].
__global__ void validate_keys(long long m, int n, int b, u64 loop_key, const int *src, const int *dst,
                              const int *cap, const int *perm, u64 *key, unsigned *val, int *bad,
                              unsigned long long *nonloop)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    unsigned long long local = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += stride) {
        int u = src[i], v = dst[i], c = cap[i];
        if (u < 0 || u >= n || v < 0 || v >= n || c < 0) {
            atomicOr(bad, 1);
            u = v = 0;
        } else if (perm) {
            u = __ldg(perm + u);
            v = __ldg(perm + v);
        }
        if (u != v) {
            key[i] = ((u64)(unsigned)u << b) | (unsigned)v;
            ++local;
        } else {
            key[i] = loop_key;
        }
        val[i] = (unsigned)i;
    }
    typedef cub::BlockReduce<unsigned long long, 256> Reduce;
    __shared__ typename Reduce::TempStorage tmp;
    local = Reduce(tmp).Sum(local);
    if (threadIdx.x == 0 && local) atomicAdd(nonloop, local);
}

// BCSR half-entries: position 2i is input arc i seen from its tail (row u,
// col v), position 2i + 1 the same arc seen from its head (row v, col u).
// The arcs sorted by (u, v) are the tail-side half-entries in order; a
// stable sort of that list by v gives the head-side ones in order, and a
// merge of the two lists by (key, position) gives every half-entry in the
// order of one stable sort by key.

// Head-side list entry: the arc's tail, its input index and its capacity.
struct InVal {
    unsigned u;
    unsigned i;
    int c;
};

// Keys and values of the head-side sort from the (u, v)-sorted arcs k < mp
// (self-loops sorted after them), and the capacities in that order (ctail,
// so that the merge reads the tail side's capacities in sequence instead of
// gathering them a second time).  Also flags (dup = 1) a parallel arc: two
// equal neighbouring keys, the only case that needs the duplicate prefix.
__global__ void in_prep(long long mp, int b, const u64 *key, const unsigned *val, const int *cap, unsigned *kin,
                        InVal *vin, int *ctail, int *dup)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const u64 mask = (1ull << b) - 1;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < mp; k += stride) {
        const u64 x = key[k];
        const unsigned i = val[k];
        const int c = cap[i];
        kin[k] = (unsigned)(x & mask);
        vin[k] = InVal{(unsigned)(x >> b), i, c};
        ctail[k] = c;
        if (k > 0 && key[k - 1] == x) *dup = 1;
    }
}

// One half-entry as the merge sees it: packed (row, col) key, position, and
// capacity (c on the tail side, -(c + 1) on the head side, c >= 0).
struct HalfRec {
    u64 k;
    unsigned p;
    int c;
};

struct HalfLess {
    __host__ __device__ bool operator()(const HalfRec &a, const HalfRec &b) const
    {
        return a.k < b.k || (a.k == b.k && a.p < b.p);
    }
};

// k-th tail-side half-entry (ctail: capacities in the (u, v) order).
struct OutHalf {
    const u64 *key;
    const unsigned *val;
    const int *ctail;
    __host__ __device__ HalfRec operator()(long long k) const
    {
        return HalfRec{key[k], 2u * val[k], ctail[k]};
    }
};

// q-th head-side half-entry.
struct InHalf {
    int b;
    const unsigned *kin;
    const InVal *vin;
    __host__ __device__ HalfRec operator()(long long q) const
    {
        const InVal x = vin[q];
        return HalfRec{((u64)kin[q] << b) | x.u, 2u * x.i + 1u, -x.c - 1};
    }
};

struct SplitHalf {
    __host__ __device__ thrust::tuple<u64, unsigned, int> operator()(const HalfRec &r) const
    {
        return thrust::make_tuple(r.k, r.p, r.c);
    }
};

// The tail-side capacity of a merged capacity entry (0 on the head side).
struct TailPart {
    __host__ __device__ int operator()(int x) const { return x > 0 ? x : 0; }
};

// Lean builds: the duplicate prefix by walking each run of equal keys from
// its head (runs are as long as the duplicates of one pair).
__global__ void run_prefix(long long len, const u64 *key, const unsigned *pos, const int *cj, int *prefix)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < len; j += stride) {
        const u64 k = key[j];
        if (j > 0 && key[j - 1] == k) continue;
        long long acc = 0;  // (a pair whose capacities exceed INT32_MAX fails the build when merged)
        for (long long i = j; i < len && key[i] == k; ++i) {
            const int x = cj[i];
            if (x < 0) continue;  // head-side half-entry
            prefix[pos[i] >> 1] = (int)acc;
            acc += x;
        }
    }
}

__global__ void scatter_prefix(long long len, const unsigned *pos, const int *pre, int *prefix)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < len; j += stride) {
        const unsigned p = pos[j];
        if ((p & 1u) == 0) prefix[p >> 1] = pre[j];
    }
}

// 1 where a run of equal keys starts (the scan's input, read on the fly).
struct RunHead {
    const u64 *key;
    __host__ __device__ unsigned operator()(long long j) const
    {
        return (j == 0 || key[j] != key[j - 1]) ? 1u : 0u;
    }
};

// slot_of = inclusive scan of run heads (1-based slot numbers).  Every
// half-entry records its slot; the head of each run (one neighbour pair seen
// from one side) writes the slot's column, sums the capacities of the run's
// tail-side half-entries into cf0 / cf (flag 2 on int32 overflow), and, when
// its slot is the last of its row r, writes r's end into off[r + 1] (off is
// zeroed before; an inclusive max-scan afterwards gives rows without slots
// the end of the row before them).  The run's head-side half-entries are the arcs col ->
// row, so their capacities sum to the paired slot's cf0: the pair's total
// must fit int32 (flag 4), since a push moves residual capacity from one slot
// to the other, and with the mirror (cfb != null) it is the initial cfb.
// Runs are short: one per (u, v), as long as the number of duplicate arcs
// between u and v.
struct RunOut {
    int *col, *cf0, *cf, *cfb;
    long long *off;
    unsigned *arc2slot;
    int *bad;
};

// Half-entry j (key k, position p, slot a; kp the key before it).
__device__ __forceinline__ void merge_one(long long j, long long len, int b, u64 k, u64 kp, unsigned p, unsigned a,
                                          const u64 *key, const int *cj, const RunOut &o)
{
    if ((p & 1u) == 0) o.arc2slot[p >> 1] = a;  // an arc's slot is that of its tail-side half-entry
    if (k == kp) return;
    o.col[a] = (int)(k & ((1ull << b) - 1));
    long long sum = 0, back = 0;
    long long i = j;
    for (; i < len && key[i] == k; ++i) {
        const int x = cj[i];
        if (x >= 0) sum += x;
        else back += -(long long)x - 1;
    }
    const long long r = (long long)(k >> b);
    if (i == len || (long long)(key[i] >> b) != r) o.off[r + 1] = (long long)a + 1;
    if (sum > 0x7fffffffLL) {
        atomicOr(o.bad, 2);
        sum = 0;
    }
    if (sum + back > 0x7fffffffLL) {
        atomicOr(o.bad, 4);
        back = 0;
    }
    o.cf0[a] = (int)sum;
    o.cf[a] = (int)sum;
    if (o.cfb) o.cfb[a] = (int)back;
}

// Half-entries start..len-1, one per thread and step.
__global__ void merge_runs(long long start, long long len, int b, const u64 *key, const unsigned *pos,
                           const unsigned *slot_of, const int *cj, RunOut o)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = start + blockIdx.x * (long long)blockDim.x + threadIdx.x; j < len; j += stride)
        merge_one(j, len, b, key[j], j == 0 ? ~0ull : key[j - 1], pos[j], slot_of[j] - 1, key, cj, o);
}

// Half-entries 0..4 * (len / 4) - 1, four consecutive ones per thread and
// step, with 16-byte loads (key, pos, slot_of 16-byte aligned).
__global__ void merge_runs4(long long len, int b, const u64 *key, const unsigned *pos, const unsigned *slot_of,
                            const int *cj, RunOut o)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n4 = len >> 2;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4; q += stride) {
        const ulonglong2 k01 = reinterpret_cast<const ulonglong2 *>(key)[2 * q];       // the run loop
        const ulonglong2 k23 = reinterpret_cast<const ulonglong2 *>(key)[2 * q + 1];   // reads these again
        const uint4 p4 = __ldcs(reinterpret_cast<const uint4 *>(pos) + q);
        const uint4 s4 = __ldcs(reinterpret_cast<const uint4 *>(slot_of) + q);
        const long long j = 4 * q;
        const u64 kp = j == 0 ? ~0ull : key[j - 1];
        merge_one(j, len, b, k01.x, kp, p4.x, s4.x - 1, key, cj, o);
        merge_one(j + 1, len, b, k01.y, k01.x, p4.y, s4.y - 1, key, cj, o);
        merge_one(j + 2, len, b, k23.x, k01.y, p4.z, s4.z - 1, key, cj, o);
        merge_one(j + 3, len, b, k23.y, k23.x, p4.w, s4.w - 1, key, cj, o);
    }
}

// BCSR reverse index: every head-side half-entry (slot a, of arc i) pairs
// a with the arc's tail-side slot arc2slot[i], both ways.  Every slot holds
// a half-entry of some arc, on one side or the other, so every slot is
// written; duplicate arcs write the same values again.
__global__ void rev_pairs(long long start, long long len, const unsigned *pos, const unsigned *slot_of,
                          const unsigned *arc2slot, unsigned *rev)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = start + blockIdx.x * (long long)blockDim.x + threadIdx.x; j < len; j += stride) {
        const unsigned p = pos[j];
        if ((p & 1u) == 0) continue;
        const unsigned a = slot_of[j] - 1, t = arc2slot[p >> 1];
        rev[a] = t;
        rev[t] = a;
    }
}

// Half-entries 0..4 * (len / 4) - 1, four consecutive ones per thread and
// step (16-byte loads of pos and slot_of): their gathers from arc2slot are
// independent, so up to four are in flight per thread.
__global__ void rev_pairs4(long long len, const unsigned *pos, const unsigned *slot_of, const unsigned *arc2slot,
                           unsigned *rev)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n4 = len >> 2;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4; q += stride) {
        const uint4 p4 = __ldcs(reinterpret_cast<const uint4 *>(pos) + q);
        const uint4 s4 = __ldcs(reinterpret_cast<const uint4 *>(slot_of) + q);
        const unsigned p[4] = {p4.x, p4.y, p4.z, p4.w};
        const unsigned a[4] = {s4.x - 1, s4.y - 1, s4.z - 1, s4.w - 1};
        unsigned t[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (p[e] & 1u) t[e] = __ldcg(arc2slot + (p[e] >> 1));
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (p[e] & 1u) {
                rev[a[e]] = t[e];
                rev[t[e]] = a[e];
            }
    }
}

// Row ends from sorted row keys: the last slot a of row r writes off[r + 1] =
// a + 1 (off zeroed before); the max-scan of close_offsets() then fills the
// rows without slots.
__global__ void row_offsets(long long S, const u64 *key, int shift, long long *off)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < S; a += stride) {
        const long long r = (long long)(key[a] >> shift);
        if (a == S - 1 || (long long)(key[a + 1] >> shift) != r) off[r + 1] = a + 1;
    }
}

// Renumbering (wbpr_options.renumber): endpoint counts per vertex, one atomic per distinct endpoint
// of a warp's 32 arcs (inputs often come sorted by tail, so a warp's tails
// repeat).  Ids are checked here, since the remap indexes by them (flag 1:
// out of range or negative capacity).  Every lane of the warp runs the same
// number of rounds.
__global__ void count_degrees_warp(long long m, int n, const int *src, const int *dst, const int *cap,
                                   unsigned *deg, int *bad)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long rounds = (m + stride - 1) / stride;
    const int lane = threadIdx.x & 31;
    for (long long q = 0; q < rounds; ++q) {
        const long long i = q * stride + blockIdx.x * (long long)blockDim.x + threadIdx.x;
        int u = -1, v = -1;
        if (i < m) {
            u = src[i];
            v = dst[i];
            if (u < 0 || u >= n || v < 0 || v >= n || cap[i] < 0) {
                atomicOr(bad, 1);
                u = v = -1;
            } else if (u == v) {
                u = v = -1;
            }
        }
        const unsigned gu = __match_any_sync(0xffffffffu, u);
        if (u >= 0 && lane == __ffs(gu) - 1) atomicAdd(deg + u, (unsigned)__popc(gu));
        const unsigned gv = __match_any_sync(0xffffffffu, v);
        if (v >= 0 && lane == __ffs(gv) - 1) atomicAdd(deg + v, (unsigned)__popc(gv));
    }
}

// Rows without slots take the end of the row before them: inclusive
// max-scan over off[0..n] (off[0] = 0), in place.
wbpr_status close_offsets_scan(long long *off, long long n, void *tmp, size_t *tmp_bytes, cudaStream_t st)
{
    cudaError_t e = cub::DeviceScan::InclusiveScan(tmp, *tmp_bytes, off, off, cuda::maximum<>(), (int64_t)(n + 1), st);
    if (e != cudaSuccess) return set_error(WBPR_ECUDA, std::string("build: offsets scan: ") + cudaGetErrorString(e));
    return WBPR_OK;
}

__global__ void iota_u32(long long len, unsigned *p)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += stride) p[i] = (unsigned)i;
}

// order[j] = the input id of new vertex j; perm is its inverse.
__global__ void invert_order(long long n, const int *order, int *perm)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += stride) perm[order[j]] = (int)j;
}

__global__ void remap_arcs(long long m, const int *perm, const int *src, const int *dst, int *rsrc, int *rdst)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += stride) {
        rsrc[i] = perm[src[i]];
        rdst[i] = perm[dst[i]];
    }
}

__global__ void fill_i64(long long len, long long *p, long long x)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += stride) p[i] = x;
}

__global__ void max_degree_kernel(int n, const long long *off, const long long *in_off,
                                  unsigned long long *out)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    unsigned long long mx = 0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += stride) {
        long long d = off[v + 1] - off[v];
        if (in_off) d += in_off[v + 1] - in_off[v];
        if ((unsigned long long)d > mx) mx = (unsigned long long)d;
    }
    typedef cub::BlockReduce<unsigned long long, 256> Reduce;
    __shared__ typename Reduce::TempStorage tmp;
    mx = Reduce(tmp).Reduce(mx, cuda::maximum<>());
    if (threadIdx.x == 0 && mx) atomicMax(out, mx);
}

__global__ void rcsr_out(long long mp, int b, const unsigned *val, const int *dst, const int *cap,
                         const u64 *key_sorted, int *col, int *cf0, int *cf, unsigned *arc2slot,
                         u64 *key_in, unsigned *val_in)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < mp; j += stride) {
        unsigned i = val[j];
        col[j] = dst[i];
        cf0[j] = cap[i];
        cf[j] = cap[i];
        arc2slot[i] = (unsigned)j;
        u64 k = key_sorted[j];
        key_in[j] = ((k & ((1ull << b) - 1)) << b) | (k >> b);
        val_in[j] = (unsigned)j;
    }
}

__global__ void rcsr_in(long long mp, int b, const u64 *key_in_sorted, const unsigned *val_in_sorted,
                        int *in_col, unsigned *flow_idx)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < mp; k += stride) {
        in_col[k] = (int)(key_in_sorted[k] & ((1ull << b) - 1));
        flow_idx[k] = val_in_sorted[k];
    }
}

// Grid of a grid-stride builder kernel: one thread per item, at most 32
// blocks of 256 per SM of the current device.
inline int grid_for(long long work)
{
    static thread_local int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
            cudaGetLastError();
            sms = 1;
        }
    }
    long long b = (work + 255) / 256;
    if (b < 1) b = 1;
    if (b > 32LL * sms) b = 32LL * sms;
    return (int)b;
}

inline int bitlen(long long x)
{
    int b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

// Scratch allocations released at the end of the build.
struct Scratch {
    struct Held {
        void *p;
        size_t bytes;
        DevFree owner;
    };
    cudaStream_t st;
    std::vector<Held> held;
    explicit Scratch(cudaStream_t s) : st(s) {}
    void *get(size_t bytes)
    {
        if (bytes == 0) bytes = 16;
        DevFree owner;
        void *p = dev_alloc(bytes, st, &owner);
        if (p) held.push_back({p, bytes, owner});
        return p;
    }
    void release(void *p)
    {
        for (size_t i = 0; i < held.size(); ++i)
            if (held[i].p == p) {
                dev_free(p, held[i].bytes, st, &held[i].owner);
                held.erase(held.begin() + (long)i);
                return;
            }
    }
    ~Scratch()
    {
        for (auto &b : held) dev_free(b.p, b.bytes, st, &b.owner);
    }
};

#define BUILD_CUDA(call)                                                               \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return set_error(WBPR_ECUDA, std::string("build: ") + #call + ": " +       \
                                             cudaGetErrorString(e_));                  \
    } while (0)

#define BUILD_ALLOC(ptr, type, count, pool)                                            \
    do {                                                                               \
        ptr = (type *)(pool).get(sizeof(type) * (size_t)(count));                      \
        if (!ptr) return set_error(WBPR_ENOMEM, "build: device allocation failed");    \
    } while (0)

#define OWN_ALLOC(ptr, type, count)                                                    \
    do {                                                                               \
        ptr = (type *)g->alloc(sizeof(type) * (size_t)(count), st);                    \
        if (!ptr) return set_error(WBPR_ENOMEM, "build: device allocation failed");    \
    } while (0)

}  // namespace

wbpr_status build_graph(wbpr_graph *g, const int *src, const int *dst, const int *cap,
                        cudaStream_t st)
{
    const long long n = g->n, m = g->m;
    Scratch pool(st);
    int *bad;
    unsigned long long *counter;
    BUILD_ALLOC(bad, int, 4, pool);
    BUILD_ALLOC(counter, unsigned long long, 4, pool);
    BUILD_CUDA(cudaMemsetAsync(bad, 0, 4 * sizeof(int), st));
    BUILD_CUDA(cudaMemsetAsync(counter, 0, 4 * sizeof(unsigned long long), st));
    // Keys pack (row, col) into 2 * kb bits.  The all-ones key would be the
    // self-loop (2^kb - 1, 2^kb - 1), so it can mark self-loops: they sort last.
    const int kb = bitlen(n - 1);
    const int end_bit = 2 * kb;
    const u64 loop_key = (1ull << end_bit) - 1;
    int h_bad = 0;
    unsigned long long h_nonloop = 0;

    // ---- optional renumbering by endpoint count, largest first ---------------
    // Vertices that many arcs point to get neighbouring ids, so the heights the
    // residual scans gather (h[col]) share sectors and stay in L2.  The solver
    // runs on the new ids; the cut side is written back in input ids, edge
    // flows are per input arc, and s, t are mapped here.
    g->s_int = g->s;
    g->t_int = g->t;
    g->order = nullptr;
    g->perm = nullptr;
    if (g->renumbered && m > 0) {
        unsigned *deg, *degs, *ids;
        BUILD_ALLOC(deg, unsigned, n, pool);
        BUILD_ALLOC(degs, unsigned, n, pool);
        BUILD_ALLOC(ids, unsigned, n, pool);
        OWN_ALLOC(g->order, int, n);
        BUILD_CUDA(cudaMemsetAsync(deg, 0, sizeof(unsigned) * (size_t)n, st));
        count_degrees_warp<<<grid_for(m), 256, 0, st>>>(m, (int)n, src, dst, cap, deg, bad);
        iota_u32<<<grid_for(n), 256, 0, st>>>(n, ids);
        BUILD_CUDA(cudaGetLastError());
        BUILD_CUDA(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
        BUILD_CUDA(cudaStreamSynchronize(st));
        if (h_bad) return set_error(WBPR_EINVAL, "build: vertex id out of range or negative capacity");
        size_t nb = 0;
        // stable: equal counts keep increasing input ids
        BUILD_CUDA(cub::DeviceRadixSort::SortPairsDescending(nullptr, nb, deg, degs, ids, (unsigned *)g->order,
                                                             (int64_t)n, 0, 32, st));
        void *t0 = pool.get(nb);
        if (!t0) return set_error(WBPR_ENOMEM, "build: device allocation failed");
        BUILD_CUDA(cub::DeviceRadixSort::SortPairsDescending(t0, nb, deg, degs, ids, (unsigned *)g->order,
                                                             (int64_t)n, 0, 32, st));
        pool.release(t0);
        pool.release(ids);
        pool.release(degs);
        pool.release(deg);
        int *perm;
        OWN_ALLOC(g->perm, int, n);
        perm = g->perm;
        invert_order<<<grid_for(n), 256, 0, st>>>(n, g->order, perm);
        if (g->layout != WBPR_BCSR) {
            // RCSR reads the renumbered endpoints more than once; BCSR's key
            // pass maps them itself
            int *rsrc, *rdst;
            BUILD_ALLOC(rsrc, int, m, pool);
            BUILD_ALLOC(rdst, int, m, pool);
            remap_arcs<<<grid_for(m), 256, 0, st>>>(m, perm, src, dst, rsrc, rdst);
            src = rsrc;
            dst = rdst;
        }
        BUILD_CUDA(cudaGetLastError());
        int st_int[2];
        BUILD_CUDA(cudaMemcpyAsync(&st_int[0], perm + g->s, sizeof(int), cudaMemcpyDeviceToHost, st));
        BUILD_CUDA(cudaMemcpyAsync(&st_int[1], perm + g->t, sizeof(int), cudaMemcpyDeviceToHost, st));
        BUILD_CUDA(cudaStreamSynchronize(st));
        g->s_int = st_int[0];
        g->t_int = st_int[1];
    }

    OWN_ALLOC(g->arc2slot, unsigned, m);
    OWN_ALLOC(g->off, long long, n + 1);
    BUILD_CUDA(cudaMemsetAsync(g->off, 0, sizeof(long long) * (size_t)(n + 1), st));
    auto close_offsets = [&](long long *o) -> wbpr_status {
        size_t nb = 0;
        wbpr_status r = close_offsets_scan(o, n, nullptr, &nb, st);
        if (r != WBPR_OK) return r;
        void *t = pool.get(nb);
        if (!t) return set_error(WBPR_ENOMEM, "build: device allocation failed");
        r = close_offsets_scan(o, n, t, &nb, st);
        pool.release(t);
        return r;
    };
    unsigned long long *h_maxdeg_dev = counter + 1;
    BUILD_CUDA(cudaMemsetAsync(g->arc2slot, 0xff, sizeof(unsigned) * (size_t)(m > 0 ? m : 1), st));

    if (g->layout == WBPR_BCSR) {
        // ---- tail-side order: the arcs sorted by (u, v) ------------------------------
        u64 *ko, *kob;
        unsigned *vo, *vob;
        BUILD_ALLOC(ko, u64, m, pool);
        BUILD_ALLOC(kob, u64, m, pool);
        BUILD_ALLOC(vo, unsigned, m, pool);
        BUILD_ALLOC(vob, unsigned, m, pool);
        if (m > 0) {
            validate_keys<<<grid_for(m), 256, 0, st>>>(m, (int)n, kb, loop_key, src, dst, cap, g->perm, ko, vo, bad,
                                                       counter);
            BUILD_CUDA(cudaGetLastError());
        }
        BUILD_CUDA(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
        BUILD_CUDA(cudaMemcpyAsync(&h_nonloop, counter, sizeof(h_nonloop), cudaMemcpyDeviceToHost, st));
        BUILD_CUDA(cudaStreamSynchronize(st));
        if (h_bad) return set_error(WBPR_EINVAL, "build: vertex id out of range or negative capacity");
        const long long mp = (long long)h_nonloop;
        g->mprime = mp;
        cub::DoubleBuffer<u64> dko(ko, kob);
        cub::DoubleBuffer<unsigned> dvo(vo, vob);
        if (m > 0) {
            size_t nb = 0;
            BUILD_CUDA(sort_pairs(g->lean, nullptr, nb, dko, dvo, (int64_t)m, 0, end_bit, st));
            void *t3 = pool.get(nb);
            if (!t3) return set_error(WBPR_ENOMEM, "build: device allocation failed");
            BUILD_CUDA(sort_pairs(g->lean, t3, nb, dko, dvo, (int64_t)m, 0, end_bit, st));
            pool.release(t3);
        }
        u64 *kos = dko.Current();
        unsigned *vos = dvo.Current();
        pool.release(kos == ko ? kob : ko);
        pool.release(vos == vo ? vob : vo);
        const long long len = 2 * mp;  // self-loops sort last and get no half-entries

        // ---- head-side order: the same arcs stably sorted by v ------------------------
        // Stable over the (u, v) order, so the result is the (v, u) order with
        // duplicates still in input order.  Tail, input index and capacity ride
        // along, so no later pass gathers them.
        int *dup = bad + 2;   // zeroed with the other flags
        unsigned *kin = nullptr, *kinb = nullptr;
        InVal *vin = nullptr, *vinb = nullptr;
        BUILD_ALLOC(kin, unsigned, mp, pool);
        BUILD_ALLOC(kinb, unsigned, mp, pool);
        BUILD_ALLOC(vin, InVal, mp, pool);
        BUILD_ALLOC(vinb, InVal, mp, pool);
        int *ctail = nullptr;
        BUILD_ALLOC(ctail, int, mp, pool);
        cub::DoubleBuffer<unsigned> dki(kin, kinb);
        cub::DoubleBuffer<InVal> dvi(vin, vinb);
        if (mp > 0) {
            in_prep<<<grid_for(mp), 256, 0, st>>>(mp, kb, kos, vos, cap, kin, vin, ctail, dup);
            BUILD_CUDA(cudaGetLastError());
            size_t nb = 0;
            BUILD_CUDA(sort_pairs(g->lean, nullptr, nb, dki, dvi, (int64_t)mp, 0, kb, st));
            void *t6 = pool.get(nb);
            if (!t6) return set_error(WBPR_ENOMEM, "build: device allocation failed");
            BUILD_CUDA(sort_pairs(g->lean, t6, nb, dki, dvi, (int64_t)mp, 0, kb, st));
            pool.release(t6);
        }
        unsigned *kis = dki.Current();
        InVal *vis = dvi.Current();
        pool.release(kis == kin ? kinb : kin);
        pool.release(vis == vin ? vinb : vin);

        // ---- both half-entries in (row, col) order: merge the two lists --------------
        // Records compare by (key, position); positions are unique (2i tail side,
        // 2i + 1 head side), so the merge is the stable sort of all half-entries
        // by key.  Outputs: sorted keys, positions, and capacities (c on the tail
        // side, -(c + 1) on the head side).
        u64 *k2s = nullptr;
        unsigned *v2s = nullptr;
        int *cj = nullptr;
        BUILD_ALLOC(k2s, u64, len, pool);
        BUILD_ALLOC(v2s, unsigned, len, pool);
        BUILD_ALLOC(cj, int, len, pool);
        if (len > 0) {
            auto in1 = thrust::make_transform_iterator(thrust::counting_iterator<long long>(0), OutHalf{kos, vos, ctail});
            auto in2 = thrust::make_transform_iterator(thrust::counting_iterator<long long>(0), InHalf{kb, kis, vis});
            auto out = thrust::make_transform_output_iterator(thrust::make_zip_iterator(k2s, v2s, cj), SplitHalf{});
            size_t nb = 0;
            BUILD_CUDA(cub::DeviceMerge::MergeKeys(nullptr, nb, in1, (int64_t)mp, in2, (int64_t)mp, out, HalfLess{},
                                                   st));
            void *t7 = pool.get(nb);
            if (!t7) return set_error(WBPR_ENOMEM, "build: device allocation failed");
            BUILD_CUDA(cub::DeviceMerge::MergeKeys(t7, nb, in1, (int64_t)mp, in2, (int64_t)mp, out, HalfLess{}, st));
            pool.release(t7);
        }
        pool.release(kis);
        pool.release(vis);
        pool.release(kos);
        pool.release(vos);
        pool.release(ctail);

        // ---- duplicate prefix (edge-flow split in input order) ------------------
        // The tail-side half-entries of duplicates of (u, v) sit in input order
        // in one run: an exclusive sum by key over their capacities.
        OWN_ALLOC(g->prefix, int, m);
        OWN_ALLOC(g->cap_in, int, m);
        if (m > 0) BUILD_CUDA(cudaMemcpyAsync(g->cap_in, cap, sizeof(int) * (size_t)m, cudaMemcpyDeviceToDevice, st));
        BUILD_CUDA(cudaMemsetAsync(g->prefix, 0, sizeof(int) * (size_t)(m > 0 ? m : 1), st));

        // ---- merge runs into slots ------------------------------------------------
        unsigned *heads;
        BUILD_ALLOC(heads, unsigned, len, pool);
        unsigned S = 0;
        if (len > 0) {
            auto flags = thrust::make_transform_iterator(thrust::counting_iterator<long long>(0), RunHead{k2s});
            size_t nb = 0;
            BUILD_CUDA(cub::DeviceScan::InclusiveSum(nullptr, nb, flags, heads, (int64_t)len, st));
            void *t4 = pool.get(nb);
            if (!t4) return set_error(WBPR_ENOMEM, "build: device allocation failed");
            BUILD_CUDA(cub::DeviceScan::InclusiveSum(t4, nb, flags, heads, (int64_t)len, st));
            pool.release(t4);
            BUILD_CUDA(cudaMemcpyAsync(&S, heads + (len - 1), sizeof(unsigned), cudaMemcpyDeviceToHost, st));
            int h_dup = 0;
            BUILD_CUDA(cudaMemcpyAsync(&h_dup, dup, sizeof(int), cudaMemcpyDeviceToHost, st));
            BUILD_CUDA(cudaStreamSynchronize(st));
            if (h_dup && g->lean) {
                run_prefix<<<grid_for(len), 256, 0, st>>>(len, k2s, v2s, cj, g->prefix);
                BUILD_CUDA(cudaGetLastError());
            } else if (h_dup) {
                // parallel arcs: each one's prefix (capacity of its earlier duplicates)
                int *pre;
                BUILD_ALLOC(pre, int, len, pool);
                auto tails = thrust::make_transform_iterator(cj, TailPart());
                size_t nb = 0;
                BUILD_CUDA(cub::DeviceScan::ExclusiveSumByKey(nullptr, nb, k2s, tails, pre, (int64_t)len,
                                                              cuda::std::equal_to<>(), st));
                void *t2 = pool.get(nb);
                if (!t2) return set_error(WBPR_ENOMEM, "build: device allocation failed");
                BUILD_CUDA(cub::DeviceScan::ExclusiveSumByKey(t2, nb, k2s, tails, pre, (int64_t)len,
                                                              cuda::std::equal_to<>(), st));
                pool.release(t2);
                scatter_prefix<<<grid_for(len), 256, 0, st>>>(len, v2s, pre, g->prefix);
                BUILD_CUDA(cudaGetLastError());
                pool.release(pre);
            }
        }
        g->slots = S;
        OWN_ALLOC(g->col, int, S);
        OWN_ALLOC(g->cf, int, S);
        OWN_ALLOC(g->cf0, int, S);
        // The reverse index and the mirrored reverse residual only when the
        // handle uses them (paper mode, use_rev = 0, saves 8 bytes per slot).
        if (g->opts.use_rev) {
            OWN_ALLOC(g->rev, unsigned, S);
            OWN_ALLOC(g->cfb, int, S);
        }
        if (S > 0) {
            const RunOut ro{g->col, g->cf0, g->cf, g->cfb, g->off, g->arc2slot, bad};
            // four half-entries per thread where the streamed arrays allow
            // 16-byte loads, the remainder (and any unaligned case) one each
            const bool a16 = ((reinterpret_cast<uintptr_t>(k2s) | reinterpret_cast<uintptr_t>(v2s) |
                               reinterpret_cast<uintptr_t>(heads)) & 15) == 0;
            const long long done = a16 ? (len & ~3LL) : 0;
            if (done) merge_runs4<<<grid_for(done / 4), 256, 0, st>>>(len, kb, k2s, v2s, heads, cj, ro);
            if (len > done)
                merge_runs<<<grid_for(len - done), 256, 0, st>>>(done, len, kb, k2s, v2s, heads, cj, ro);
            BUILD_CUDA(cudaGetLastError());
            pool.release(cj);
            if (g->rev) {
                if (done) rev_pairs4<<<grid_for(done / 4), 256, 0, st>>>(len, v2s, heads, g->arc2slot, g->rev);
                if (len > done)
                    rev_pairs<<<grid_for(len - done), 256, 0, st>>>(done, len, v2s, heads, g->arc2slot, g->rev);
            }
            BUILD_CUDA(cudaGetLastError());
            wbpr_status rc = close_offsets(g->off);
            if (rc != WBPR_OK) return rc;
            BUILD_CUDA(cudaGetLastError());
        } else {
            fill_i64<<<grid_for(n + 1), 256, 0, st>>>(n + 1, g->off, 0);
            BUILD_CUDA(cudaGetLastError());
        }
        max_degree_kernel<<<grid_for(n), 256, 0, st>>>((int)n, g->off, nullptr, h_maxdeg_dev);
        BUILD_CUDA(cudaGetLastError());
    } else {
        // ---- RCSR: arcs sorted by (src, dst); CUB radix sort is stable ----------------
        u64 *key1, *key1b;
        unsigned *val1, *val1b;
        BUILD_ALLOC(key1, u64, m, pool);
        BUILD_ALLOC(key1b, u64, m, pool);
        BUILD_ALLOC(val1, unsigned, m, pool);
        BUILD_ALLOC(val1b, unsigned, m, pool);
        if (m > 0) {
            validate_keys<<<grid_for(m), 256, 0, st>>>(m, (int)n, kb, loop_key, src, dst, cap, nullptr, key1, val1,
                                                       bad, counter);
            BUILD_CUDA(cudaGetLastError());
        }
        BUILD_CUDA(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
        BUILD_CUDA(cudaMemcpyAsync(&h_nonloop, counter, sizeof(h_nonloop), cudaMemcpyDeviceToHost, st));
        BUILD_CUDA(cudaStreamSynchronize(st));
        if (h_bad) return set_error(WBPR_EINVAL, "build: vertex id out of range or negative capacity");
        const long long mp = (long long)h_nonloop;
        g->mprime = mp;
        cub::DoubleBuffer<u64> dk(key1, key1b);
        cub::DoubleBuffer<unsigned> dv(val1, val1b);
        if (m > 0) {
            size_t nb = 0;
            BUILD_CUDA(sort_pairs(g->lean, nullptr, nb, dk, dv, (int64_t)m, 0, end_bit, st));
            void *t1 = pool.get(nb);
            if (!t1) return set_error(WBPR_ENOMEM, "build: device allocation failed");
            BUILD_CUDA(sort_pairs(g->lean, t1, nb, dk, dv, (int64_t)m, 0, end_bit, st));
            pool.release(t1);
        }
        u64 *ks = dk.Current();
        unsigned *vs = dv.Current();
        pool.release(ks == key1 ? key1b : key1);
        pool.release(vs == val1 ? val1b : val1);
        g->slots = mp;
        OWN_ALLOC(g->col, int, mp);
        OWN_ALLOC(g->cf, int, mp);
        OWN_ALLOC(g->cf0, int, mp);
        OWN_ALLOC(g->bf, int, mp);
        OWN_ALLOC(g->in_off, long long, n + 1);
        OWN_ALLOC(g->in_col, int, mp);
        OWN_ALLOC(g->flow_idx, unsigned, mp);
        u64 *kin, *kinb;
        unsigned *vin, *vinb;
        BUILD_ALLOC(kin, u64, mp, pool);
        BUILD_ALLOC(kinb, u64, mp, pool);
        BUILD_ALLOC(vin, unsigned, mp, pool);
        BUILD_ALLOC(vinb, unsigned, mp, pool);
        if (mp > 0) {
            rcsr_out<<<grid_for(mp), 256, 0, st>>>(mp, kb, vs, dst, cap, ks, g->col, g->cf0, g->cf,
                                                   g->arc2slot, kin, vin);
            BUILD_CUDA(cudaGetLastError());
            BUILD_CUDA(cudaMemsetAsync(g->bf, 0, sizeof(int) * (size_t)mp, st));
            row_offsets<<<grid_for(mp), 256, 0, st>>>(mp, ks, kb, g->off);
            BUILD_CUDA(cudaGetLastError());
            wbpr_status rc = close_offsets(g->off);
            if (rc != WBPR_OK) return rc;
            cub::DoubleBuffer<u64> dki(kin, kinb);
            cub::DoubleBuffer<unsigned> dvi(vin, vinb);
            size_t nb = 0;
            BUILD_CUDA(sort_pairs(g->lean, nullptr, nb, dki, dvi, (int64_t)mp, 0, end_bit, st));
            void *t5 = pool.get(nb);
            if (!t5) return set_error(WBPR_ENOMEM, "build: device allocation failed");
            BUILD_CUDA(sort_pairs(g->lean, t5, nb, dki, dvi, (int64_t)mp, 0, end_bit, st));
            pool.release(t5);
            rcsr_in<<<grid_for(mp), 256, 0, st>>>(mp, kb, dki.Current(), dvi.Current(), g->in_col, g->flow_idx);
            BUILD_CUDA(cudaGetLastError());
            BUILD_CUDA(cudaMemsetAsync(g->in_off, 0, sizeof(long long) * (size_t)(n + 1), st));
            row_offsets<<<grid_for(mp), 256, 0, st>>>(mp, dki.Current(), kb, g->in_off);
            BUILD_CUDA(cudaGetLastError());
            rc = close_offsets(g->in_off);
            if (rc != WBPR_OK) return rc;
        } else {
            fill_i64<<<grid_for(n + 1), 256, 0, st>>>(n + 1, g->off, 0);
            fill_i64<<<grid_for(n + 1), 256, 0, st>>>(n + 1, g->in_off, 0);
            BUILD_CUDA(cudaGetLastError());
        }
        max_degree_kernel<<<grid_for(n), 256, 0, st>>>((int)n, g->off, g->in_off, h_maxdeg_dev);
        BUILD_CUDA(cudaGetLastError());
    }
    unsigned long long h_maxdeg = 0;
    BUILD_CUDA(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    BUILD_CUDA(cudaMemcpyAsync(&h_maxdeg, h_maxdeg_dev, sizeof(h_maxdeg), cudaMemcpyDeviceToHost, st));
    BUILD_CUDA(cudaStreamSynchronize(st));
    if (h_bad) return set_error(WBPR_EOVERFLOW, "build: a merged pair's capacity exceeds INT32_MAX");
    g->max_degree = (int64_t)h_maxdeg;
    return WBPR_OK;
}

}  // namespace wbpr
