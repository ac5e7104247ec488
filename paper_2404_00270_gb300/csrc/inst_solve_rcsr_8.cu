// One variant of the persistent solver kernel: layout RCSR, small tiles of 8 lanes.
#include "solver_impl.cuh"

namespace wbpr {
void *solve_kernel_rcsr_8() { return (void *)solve_kernel<kRCSR, 8>; }
}  // namespace wbpr
