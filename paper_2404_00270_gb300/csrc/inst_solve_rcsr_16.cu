// One variant of the persistent solver kernel: layout RCSR, small tiles of 16 lanes.
#include "solver_impl.cuh"

namespace wbpr {
void *solve_kernel_rcsr_16() { return (void *)solve_kernel<kRCSR, 16>; }
}  // namespace wbpr
