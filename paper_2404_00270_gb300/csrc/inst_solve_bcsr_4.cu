// One variant of the persistent solver kernel: layout BCSR, small tiles of 4 lanes.
#include "solver_impl.cuh"

namespace wbpr {
void *solve_kernel_bcsr_4() { return (void *)solve_kernel<kBCSR, 4>; }
}  // namespace wbpr
