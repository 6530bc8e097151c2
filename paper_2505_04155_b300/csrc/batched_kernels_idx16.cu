// batched_kernels_idx16.cu -- the persistent batched kernel (batched.cuh) for
// matrices with int16 column offsets.
// the host unit (ampcg.cu) defines the non-template kernels
#define AMPCG_INSTANTIATION_UNIT
#include "batched.cuh"
#include "kernel_table.h"

namespace ampcg {
const void* batched_kernel_idx16() { return (const void*)k_batched<1>; }
}  // namespace ampcg
