// loop_none_plain.cu -- k_loop variants: no preconditioner, four grid barriers per iteration.
#include "loop_kernels.cuh"

namespace ampcg {
const void* loop_kernel_none_plain(int uz, int ur, int it) { return loop_table<M_NONE, false>(uz, ur, it); }
}  // namespace ampcg
