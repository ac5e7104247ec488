// The persistent server kernel for layout BCSR.
#include "solver_impl.cuh"

namespace wbpr {
void *server_kernel_bcsr() { return (void *)server_kernel<kBCSR, 8>; }
}  // namespace wbpr
