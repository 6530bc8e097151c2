// loop_spmv.cu -- the persistent kernel's staged SpMV on its own
// (k_spmv_loop_step), for parity tests of that code path.
// the host unit (ampcg.cu) defines the non-template kernels
#define AMPCG_INSTANTIATION_UNIT
#include "kernel_table.h"
#include "kernels.cuh"

namespace ampcg {
template <int IT>
static const void* loop_spmv_table(int uz, int ur) {
  switch (2 * uz + ur) {
    case 0: return (const void*)k_spmv_loop_step<P64, P64, IT>;
    case 1: return (const void*)k_spmv_loop_step<P64, P32, IT>;
    case 2: return (const void*)k_spmv_loop_step<P32, P64, IT>;
    case 3: return (const void*)k_spmv_loop_step<P32, P32, IT>;
    case 4: return (const void*)k_spmv_loop_step<P16, P64, IT>;
    case 5: return (const void*)k_spmv_loop_step<P16, P32, IT>;
  }
  return nullptr;
}
const void* loop_spmv_kernel(int uz, int ur, int it) {
  return it ? loop_spmv_table<1>(uz, ur) : loop_spmv_table<0>(uz, ur);
}
}  // namespace ampcg
