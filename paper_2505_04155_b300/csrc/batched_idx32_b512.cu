// batched_idx32_b512.cu -- the persistent batched kernel (batched.cuh) for
// matrices with int32 column indices, blocks of 512 threads.
// the host unit (ampcg.cu) defines the non-template kernels
#define AMPCG_INSTANTIATION_UNIT
#include "batched.cuh"
#include "kernel_table.h"

namespace ampcg {
const void* batched_kernel_idx32_b512() { return (const void*)k_batched<0, 512>; }
}  // namespace ampcg
