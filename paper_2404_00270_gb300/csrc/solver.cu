// Kernel dispatch and launches.  The solver's device code is in
// solver_impl.cuh; its kernel variants are instantiated in inst_*.cu.
#include <stdint.h>

#include "wbpr_internal.cuh"

namespace wbpr {

// defined in inst_*.cu
void *solve_kernel_bcsr_4();
void *solve_kernel_bcsr_8();
void *solve_kernel_bcsr_16();
void *solve_kernel_rcsr_4();
void *solve_kernel_rcsr_8();
void *solve_kernel_rcsr_16();
void *server_kernel_bcsr();
void *server_kernel_rcsr();

namespace {

// Edge flows in input order.  BCSR: the merged pair's net flow u -> v is
// cf0(a) - cf(a); when positive it is split over the duplicate input arcs
// u -> v greedily in input order (prefix = capacity of earlier duplicates).
// RCSR: the flow of arc j is its backward residual bf(j).
__global__ void edge_flow_kernel(int layout, long long m, const unsigned *arc2slot,
                                 const int *cf0, const int *cf, const int *bf, const int *prefix,
                                 const int *cap_in, int *edge_flow)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += stride) {
        unsigned a = arc2slot[i];
        int f = 0;
        if (a != 0xffffffffu) {
            if (layout == kBCSR) {
                long long net = (long long)cf0[a] - (long long)cf[a];
                if (net > 0) {
                    long long x = net - prefix[i];
                    if (x < 0) x = 0;
                    if (x > cap_in[i]) x = cap_in[i];
                    f = (int)x;
                }
            } else {
                f = bf[a];
            }
        }
        edge_flow[i] = f;
    }
}

}  // namespace

static void *pick_server_kernel(int layout)
{
    return layout == kBCSR ? server_kernel_bcsr() : server_kernel_rcsr();
}

// An SM's split between L1 and shared memory is fixed while any block runs
// on it.  A server that admits builds while it is resident (build_room)
// asks for the largest shared-memory carveout, so that the builds' blocks
// (sort and scan tiles of up to 34 KB in a lean build) find shared memory
// beside its blocks; with the default carveout the split chosen for the
// server's own blocks left too little, and builds waited for the server to
// exit.  A batch, which builds nothing while its server runs, keeps the
// default (more L1).
static cudaError_t server_carveout(void *k, bool build_room)
{
    return cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                build_room ? (int)cudaSharedmemCarveoutMaxShared : (int)cudaSharedmemCarveoutDefault);
}

cudaError_t server_max_blocks_per_sm(int layout, int *blocks, bool build_room)
{
    void *k = pick_server_kernel(layout);
    cudaError_t e = server_carveout(k, build_room);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, kBlock, 0);
}

cudaError_t server_launch(int layout, int grid, const ServerDesc &d, cudaStream_t stream, bool build_room)
{
    ServerDesc local = d;
    void *args[] = {&local};
    void *k = pick_server_kernel(layout);
    cudaError_t e = server_carveout(k, build_room);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kBlock), args, 0, stream);
}

static void *pick_kernel(int layout, int small_tile)
{
    if (layout == kBCSR) {
        if (small_tile == 4) return solve_kernel_bcsr_4();
        if (small_tile == 16) return solve_kernel_bcsr_16();
        return solve_kernel_bcsr_8();
    }
    if (small_tile == 4) return solve_kernel_rcsr_4();
    if (small_tile == 16) return solve_kernel_rcsr_16();
    return solve_kernel_rcsr_8();
}

// A launch with the hub-chunk stage uses 16.8 KB of static and 32 KB of
// dynamic shared memory per block: more than the 48 KB a kernel gets without
// opting in, so the kernel opts in to that much dynamic shared memory, and
// asks for the largest shared-memory carveout so that four such blocks fit
// on an SM (a cooperative launch is sized from this occupancy).
static cudaError_t set_carveout(void *kernel, size_t dyn_smem)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                dyn_smem ? (int)cudaSharedmemCarveoutMaxShared : (int)cudaSharedmemCarveoutDefault);
}

cudaError_t solver_max_blocks_per_sm(int layout, int small_tile, int *blocks, size_t dyn_smem)
{
    void *k = pick_kernel(layout, small_tile);
    cudaError_t e = set_carveout(k, dyn_smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, kBlock, dyn_smem);
}

cudaError_t solver_launch(int layout, int small_tile, int grid, const Params &p,
                          cudaStream_t stream, size_t dyn_smem)
{
    Params local = p;
    void *args[] = {&local};
    void *k = pick_kernel(layout, small_tile);
    cudaError_t e = set_carveout(k, dyn_smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kBlock), args, dyn_smem, stream);
}

cudaError_t launch_edge_flow(int layout, long long m, const unsigned *arc2slot, const int *cf0,
                             const int *cf, const int *bf, const int *prefix, const int *cap_in,
                             int *edge_flow, cudaStream_t stream)
{
    if (m <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        sms = 1;
    }
    long long blocks = (m + 255) / 256;
    if (blocks > 16LL * sms) blocks = 16LL * sms;   // grid-stride: 16 blocks of 256 per SM
    edge_flow_kernel<<<(int)blocks, 256, 0, stream>>>(layout, m, arc2slot, cf0, cf, bf, prefix,
                                                      cap_in, edge_flow);
    return cudaGetLastError();
}

}  // namespace wbpr
