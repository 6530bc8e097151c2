// loop_kernels.cuh -- the table of k_loop variants for one preconditioner and
// one update form; included by the loop_*.cu translation units only.
#pragma once
// the host unit (ampcg.cu) defines the non-template kernels
#define AMPCG_INSTANTIATION_UNIT
#include "kernel_table.h"
#include "kernels.cuh"

namespace ampcg {

template <int MT, bool F>
const void* loop_table(int uz, int ur, int it) {
  const int ph = 2 * uz + ur;
  if (it) {
    switch (ph) {
      case 0: return (const void*)k_loop<P64, P64, MT, 1, F>;
      case 1: return (const void*)k_loop<P64, P32, MT, 1, F>;
      case 2: return (const void*)k_loop<P32, P64, MT, 1, F>;
      case 3: return (const void*)k_loop<P32, P32, MT, 1, F>;
      case 4: return (const void*)k_loop<P16, P64, MT, 1, F>;
      case 5: return (const void*)k_loop<P16, P32, MT, 1, F>;
    }
  } else {
    switch (ph) {
      case 0: return (const void*)k_loop<P64, P64, MT, 0, F>;
      case 1: return (const void*)k_loop<P64, P32, MT, 0, F>;
      case 2: return (const void*)k_loop<P32, P64, MT, 0, F>;
      case 3: return (const void*)k_loop<P32, P32, MT, 0, F>;
      case 4: return (const void*)k_loop<P16, P64, MT, 0, F>;
      case 5: return (const void*)k_loop<P16, P32, MT, 0, F>;
    }
  }
  return nullptr;
}

}  // namespace ampcg
