// loop_jacobi_plain.cu -- k_loop variants: Jacobi preconditioner, four grid barriers per iteration.
#include "loop_kernels.cuh"

namespace ampcg {
const void* loop_kernel_jacobi_plain(int uz, int ur, int it) { return loop_table<M_JACOBI, false>(uz, ur, it); }
}  // namespace ampcg
