// The persistent server kernel for layout RCSR.
#include "solver_impl.cuh"

namespace wbpr {
void *server_kernel_rcsr() { return (void *)server_kernel<kRCSR, 8>; }
}  // namespace wbpr
