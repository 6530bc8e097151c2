// batched_kernels_idx32.cu -- the persistent batched kernel (batched.cuh) for
// matrices with int32 column indices.
// the host unit (ampcg.cu) defines the non-template kernels
#define AMPCG_INSTANTIATION_UNIT
#include "batched.cuh"
#include "kernel_table.h"

namespace ampcg {
const void* batched_kernel_idx32() { return (const void*)k_batched<0>; }
}  // namespace ampcg
