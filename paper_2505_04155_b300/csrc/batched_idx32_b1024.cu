// batched_idx32_b1024.cu -- the persistent batched kernel (batched.cuh) for
// matrices with int32 column indices, blocks of 1024 threads.
// the host unit (ampcg.cu) defines the non-template kernels
#define AMPCG_INSTANTIATION_UNIT
#include "batched.cuh"
#include "kernel_table.h"

namespace ampcg {
const void* batched_kernel_idx32_b1024() { return (const void*)k_batched<0, 1024>; }
}  // namespace ampcg
