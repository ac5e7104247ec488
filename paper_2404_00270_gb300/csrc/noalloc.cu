// Allocation-free maximum flow for small graphs given in the BCSR layout.
//
// Some callers may not allocate device memory while they run: code executing
// inside a host framework's execution phase that forbids allocation (for
// example a plugin's enqueue step), real-time loops whose device memory budget
// is fixed up front, or embedders that own no CUDA allocator.  For them this
// file keeps the solver's whole working set in one file-scope device array of
// fixed size, so wbpr_maxflow_bcsr_noalloc() calls no cudaMalloc, cudaFree or
// allocating library routine.  The price: the array is held on every GPU that
// loads the library until the process exits, graphs are limited to the sizes
// below, and all calls share the one array.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <string>

#include "handle.h"
#include "wbpr.h"

namespace wbpr {
namespace {

constexpr long long kMaxN = WBPR_NOALLOC_MAX_VERTICES;
constexpr long long kMaxSlots = WBPR_NOALLOC_MAX_SLOTS;
constexpr int kMaxGrid = 1024;

// Scratch layout (byte offsets, each 256-aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffCf = 0;
constexpr size_t kOffCfb = align256(kOffCf + 4 * kMaxSlots);
constexpr size_t kOffE = align256(kOffCfb + 4 * kMaxSlots);
constexpr size_t kOffH = align256(kOffE + 8 * kMaxN);
constexpr size_t kOffDead = align256(kOffH + 4 * kMaxN);
constexpr size_t kOffCount = align256(kOffDead + kMaxN);
constexpr size_t kOffQ = align256(kOffCount + 4 * (kMaxN + 1));
constexpr size_t kOffHubStart = align256(kOffQ + 6 * 4 * kMaxN);
constexpr long long kMaxChunks = hub_chunk_entries(kMaxN, kMaxSlots, kBCSR);
constexpr size_t kOffHubChunk = align256(kOffHubStart + 2 * 4 * kMaxN);
constexpr size_t kOffHubE0 = align256(kOffHubChunk + 2 * 4 * kMaxChunks);
constexpr size_t kOffHubRem = align256(kOffHubE0 + 2 * 8 * kMaxN);
constexpr size_t kOffHubAux = align256(kOffHubRem + 2 * 8 * kMaxN);
constexpr size_t kOffHubDone = align256(kOffHubAux + 2 * 8 * kMaxN);
constexpr size_t kOffCtl = align256(kOffHubDone + 2 * 4 * kMaxN);
constexpr size_t kOffStats = align256(kOffCtl + sizeof(Ctl));
constexpr size_t kScratchBytes = align256(kOffStats + 8 * (size_t)kStatCount * kMaxGrid);

static_assert(kScratchBytes <= (size_t)16 << 20, "no-alloc scratch must stay modest");

// The whole working set of the allocation-free solver.  Shared by every call
// in the process; keeps the last call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
unsigned char *g_scratch_ptr[64] = {nullptr};  // device address per device ordinal

// Once per device, with that device current: the device address of the array.
wbpr_status scratch_address(int device, unsigned char **out)
{
    if (device < 0 || device >= 64) return set_error(WBPR_ECUDA, "noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return set_error(WBPR_ECUDA, std::string("noalloc: cudaGetSymbolAddress failed: ") +
                                             cudaGetErrorString(e));
        }
        g_scratch_ptr[device] = (unsigned char *)p;
    }
    *out = g_scratch_ptr[device];
    return WBPR_OK;
}

// Checks the caller's BCSR arrays before a solve trusts them: off[0] = 0,
// off[n] = slots, rows non-decreasing, neighbours in [0, n), capacities >= 0,
// and rev[] a pairing of slots whose partner lies in the neighbour's row and
// points back to the owner.  Any failure stores WBPR_EINVAL in *err.  Reads
// only off[0..n] and the [slots] arrays; the row of a slot is found by binary
// search over off.
__global__ void noalloc_check_kernel(int n, long long slots, const long long *off, const int *col,
                                     const int *cap, const unsigned *rev, int *err)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0 && (off[0] != 0 || off[n] != slots)) atomicCAS(err, 0, (int)WBPR_EINVAL);
    for (long long v = tid; v < n; v += stride)
        if (off[v] > off[v + 1]) atomicCAS(err, 0, (int)WBPR_EINVAL);
    if (off[0] != 0 || off[n] != slots) return;
    for (long long k = tid; k < slots; k += stride) {
        const int w = col[k];
        const unsigned r = rev[k];
        if (w < 0 || w >= n || cap[k] < 0 || (long long)r >= slots) {
            atomicCAS(err, 0, (int)WBPR_EINVAL);
            continue;
        }
        // owner row of k: the last v with off[v] <= k
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (int)(((long long)lo + hi + 1) >> 1);
            if (off[mid] <= k) lo = mid;
            else hi = mid - 1;
        }
        if (rev[r] != (unsigned)k || col[r] != lo || (long long)r < off[w] || (long long)r >= off[w + 1])
            atomicCAS(err, 0, (int)WBPR_EINVAL);
    }
}

}  // namespace
}  // namespace wbpr

using namespace wbpr;

extern "C" wbpr_status wbpr_maxflow_bcsr_noalloc(int32_t n, int64_t slots, int32_t s, int32_t t,
                                                 const int64_t *off, const int32_t *col,
                                                 const int32_t *cap, const uint32_t *rev,
                                                 wbpr_stream_t stream, int64_t *d_value,
                                                 int32_t *d_residual)
{
    if (n < 2 || s < 0 || t < 0 || s >= n || t >= n || s == t || slots < 0)
        return set_error(WBPR_EINVAL, "wbpr_maxflow_bcsr_noalloc: need n >= 2, slots >= 0, 0 <= s,t < n, s != t");
    if (n > kMaxN || slots > kMaxSlots)
        return set_error(WBPR_EINVAL, "wbpr_maxflow_bcsr_noalloc: graph larger than the fixed scratch (at most " +
                                          std::to_string(kMaxN) + " vertices and " + std::to_string(kMaxSlots) +
                                          " BCSR slots)");
    if (!off || !d_value || (slots > 0 && (!col || !cap || !rev)))
        return set_error(WBPR_EINVAL, "wbpr_maxflow_bcsr_noalloc: NULL pointer");
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return set_error(WBPR_ECUDA, "wbpr_maxflow_bcsr_noalloc: no CUDA device");
    }
    unsigned char *base = nullptr;
    wbpr_status rc = scratch_address(device, &base);
    if (rc != WBPR_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;

    int num_sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device);
    if (solver_max_blocks_per_sm(kBCSR, 8, &per_sm) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return set_error(WBPR_ECUDA, "wbpr_maxflow_bcsr_noalloc: occupancy query failed");
    }
    long long grid = (n + 4LL * kBlock - 1) / (4LL * kBlock);
    if (grid < num_sms) grid = num_sms;
    if (grid > (long long)per_sm * num_sms) grid = (long long)per_sm * num_sms;
    if (grid > kMaxGrid) grid = kMaxGrid;

    Params p;
    memset(&p, 0, sizeof(p));
    p.g.n = n;
    p.g.s = s;
    p.g.t = t;
    p.g.slots = slots;
    p.g.off = (const long long *)off;
    p.g.col = col;
    p.g.cf = (int *)(base + kOffCf);
    p.g.cf0 = cap;
    p.g.rev = rev;
    p.g.cfb = (int *)(base + kOffCfb);
    p.st.e = (long long *)(base + kOffE);
    p.st.h = (int *)(base + kOffH);
    p.st.dead = base + kOffDead;
    p.st.count = (int *)(base + kOffCount);
    for (int a = 0; a < 2; ++a) {
        for (int k = 0; k < kClasses; ++k) p.st.q[a][k] = (int *)(base + kOffQ) + (size_t)(a * kClasses + k) * kMaxN;
        p.st.hub_start[a] = (unsigned *)(base + kOffHubStart) + (size_t)a * kMaxN;
        p.st.hub_chunk[a] = (unsigned *)(base + kOffHubChunk) + (size_t)a * kMaxChunks;
        p.st.hub_e0[a] = (long long *)(base + kOffHubE0) + (size_t)a * kMaxN;
        p.st.hub_rem[a] = (long long *)(base + kOffHubRem) + (size_t)a * kMaxN;
        p.st.hub_aux[a] = (unsigned long long *)(base + kOffHubAux) + (size_t)a * kMaxN;
        p.st.hub_done[a] = (unsigned *)(base + kOffHubDone) + (size_t)a * kMaxN;
    }
    p.st.ctl = (Ctl *)(base + kOffCtl);
    p.st.bstats = (long long *)(base + kOffStats);
    wbpr_options o;
    wbpr_default_options(&o);
    p.mode = kModePreflow | kModePhase1;
    p.g.layout_tag = kBCSR;
    p.mirror_gather = 1;                     // the scratch may hold another graph's residuals
    p.gr_ratio = o.gr_ratio;                 // the time-balanced trigger of wbpr_maxflow,
    p.cycle = o.gr_ratio > 0.f ? 1000 : 16;  // with its automatic cycle cap
    p.gap = o.gap;
    p.use_rev = 1;
    p.multi_push = o.multi_push;
    p.small_max = o.small_max_degree;
    p.warp_max = o.warp_max_degree;
    p.bottom_up = o.bottom_up;
    p.bottom_up_min = o.bottom_up_min;
    p.bottom_up_edges = 0;                   // the automatic rule's choice below 2^21 vertices
    p.max_iterations = o.max_iterations;
    p.timeout_ns = (unsigned long long)o.barrier_timeout_ms * 1000000ull;

    // The control block must start at zero; everything else is reset by the kernel.
    // The caller's arrays are checked first (the error word of the control block).
    int err = 0;
    cudaError_t e = cudaMemsetAsync(p.st.ctl, 0, sizeof(Ctl), st);
    if (e == cudaSuccess) {
        long long cb = (slots > n ? slots : n) / 256 + 1;
        if (cb > 4LL * num_sms) cb = 4LL * num_sms;
        noalloc_check_kernel<<<(int)cb, 256, 0, st>>>(n, slots, (const long long *)off, col, cap, rev,
                                                      &p.st.ctl->err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &p.st.ctl->err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(WBPR_ECUDA, std::string("wbpr_maxflow_bcsr_noalloc: ") + cudaGetErrorString(e));
    }
    if (err != 0)
        return set_error(WBPR_EINVAL, "wbpr_maxflow_bcsr_noalloc: malformed BCSR arrays (offsets, neighbour ids, "
                                      "capacities or reverse slots)");
    if (e == cudaSuccess) e = solver_launch(kBCSR, 8, (int)grid, p, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_value, p.st.e + t, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && d_residual && slots > 0)
        e = cudaMemcpyAsync(d_residual, p.g.cf, sizeof(int32_t) * (size_t)slots, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &p.st.ctl->err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(WBPR_ECUDA, std::string("wbpr_maxflow_bcsr_noalloc: ") + cudaGetErrorString(e));
    }
    if (err != 0) return set_error((wbpr_status)err, "wbpr_maxflow_bcsr_noalloc: device solve gave up");
    return WBPR_OK;
}
