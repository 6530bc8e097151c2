// loop_none_fused.cu -- k_loop variants: no preconditioner, update step that also forms z_{k+1} and rho_{k+1} (three grid barriers per iteration).
#include "loop_kernels.cuh"

namespace ampcg {
const void* loop_kernel_none_fused(int uz, int ur, int it) { return loop_table<M_NONE, true>(uz, ur, it); }
}  // namespace ampcg
