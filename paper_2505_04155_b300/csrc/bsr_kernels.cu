// bsr_kernels.cu -- the block-row kernels for 3 x 3 block matrices (bsr.cuh).
// the host unit (ampcg.cu) defines the non-template kernels
#define AMPCG_INSTANTIATION_UNIT
#include "bsr.cuh"
#include "kernel_table.h"

namespace ampcg {

const void* bsr_spmv_kernel(int uz, int ur) {
  switch (2 * uz + ur) {
    case 0: return (const void*)k_bspmv<P64, P64>;
    case 1: return (const void*)k_bspmv<P64, P32>;
    case 2: return (const void*)k_bspmv<P32, P64>;
    case 3: return (const void*)k_bspmv<P32, P32>;
    case 4: return (const void*)k_bspmv<P16, P64>;
    case 5: return (const void*)k_bspmv<P16, P32>;
  }
  return nullptr;
}

const void* bsr_cheb_kernel(int uz, int ur) {
  switch (2 * uz + ur) {
    case 0: return (const void*)k_bcheb_step<P64, P64>;
    case 1: return (const void*)k_bcheb_step<P64, P32>;
    case 2: return (const void*)k_bcheb_step<P32, P64>;
    case 3: return (const void*)k_bcheb_step<P32, P32>;
    case 4: return (const void*)k_bcheb_step<P16, P64>;
    case 5: return (const void*)k_bcheb_step<P16, P32>;
  }
  return nullptr;
}

const void* bsr_spmv_step_kernel(int ur) {
  return ur == P64 ? (const void*)k_bspmv_step<P64> : (const void*)k_bspmv_step<P32>;
}

}  // namespace ampcg
