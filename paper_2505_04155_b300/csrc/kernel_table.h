// kernel_table.h -- addresses of the kernels that live in their own
// translation units (the persistent iteration kernel's 48 variants, the
// loop kernel's SpMV step, the batched kernel), so that the library's files
// compile in parallel.  Each of those files instantiates its kernels and
// hands out their host-side addresses here; the host code launches them
// through these addresses (cudaLaunchKernel, graph kernel nodes) and never
// instantiates them itself.
#pragma once

namespace ampcg {

// k_loop<u_z, u_r, mt, it, fused> (loop_kernels.cuh): u_z in {0,1,2}, u_r in
// {0,1}, mt in {M_NONE, M_JACOBI}, it = 1 for int16 column offsets.
const void* loop_kernel(int uz, int ur, int mt, int it, bool fused);
const void* loop_kernel_none_plain(int uz, int ur, int it);
const void* loop_kernel_none_fused(int uz, int ur, int it);
const void* loop_kernel_jacobi_plain(int uz, int ur, int it);
const void* loop_kernel_jacobi_fused(int uz, int ur, int it);

// k_spmv_loop_step<u_z, u_r, it>
const void* loop_spmv_kernel(int uz, int ur, int it);

// k_batched<it, bs>, bs = 1024 or 512 threads
const void* batched_kernel(int it, int bs);
const void* batched_kernel_idx32_b1024();
const void* batched_kernel_idx32_b512();
const void* batched_kernel_idx16_b1024();
const void* batched_kernel_idx16_b512();

// block-row kernels for 3 x 3 block matrices (bsr.cuh): k_bspmv<u_z, u_r>,
// k_bcheb_step<u_z, u_r>, k_bspmv_step<u_r>
const void* bsr_spmv_kernel(int uz, int ur);
const void* bsr_cheb_kernel(int uz, int ur);
const void* bsr_spmv_step_kernel(int ur);

}  // namespace ampcg
