// One variant of the persistent solver kernel: layout BCSR, small tiles of 8 lanes.
#include "solver_impl.cuh"

namespace wbpr {
void *solve_kernel_bcsr_8() { return (void *)solve_kernel<kBCSR, 8>; }
}  // namespace wbpr
