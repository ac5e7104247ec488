// One variant of the persistent solver kernel: layout RCSR, small tiles of 4 lanes.
#include "solver_impl.cuh"

namespace wbpr {
void *solve_kernel_rcsr_4() { return (void *)solve_kernel<kRCSR, 4>; }
}  // namespace wbpr
