// batched.cuh -- many independent small systems in one persistent launch.
//
// A block of 1024 threads runs the whole of Alg. 3 for one system at a time
// (initial residual, selector, scale + precondition, direction, SpMV,
// updates, stopping test, FP64 verification and replacement), with block
// reductions and the system's state in shared memory, so an iteration costs
// block barriers instead of kernel launches and grid-wide reductions.  Blocks
// take systems from a queue ordered by decreasing size (longest first) and
// run until the queue is empty.  The row and element loops are the
// single-system solver's (kernels.cuh) over the block's threads; only the
// reduction order differs, so iterates agree with a single-system solve to
// rounding.  The only waits are __syncthreads.
//
// Measured on the 512-system workload: splitting the larger systems over a
// cluster of 2, 4 or 8 blocks (distributed-shared-memory reductions, cluster
// barriers) was 18-80% slower than one block per system with the queue.
#pragma once
#include "kernels.cuh"

namespace ampcg {

// One system of a batch: its matrix, buffers and histories (from its
// context), where b and x live, and where its outcome goes.
struct BatchSys {
  Sell A;
  Bufs B;
  int64_t n;
  int mt;                  // M_NONE or M_JACOBI
  const double* b;         // device; copied into bbuf (= B.b) by the block
  double* x;               // device, in/out; copied to and from B.x
  double* bbuf;            // the context's padded right-hand-side buffer
  double* delta_hist;      // [maxit + 2]
  unsigned char* prec_hist;
};

// Outcome of one system.
struct BatchOut {
  int iters, status, refreshes, switch_iter[3];
  double true_relres, updated_relres, nb;
};

// Block sizes of the batched kernel: 1024 threads (one system per SM) or 512
// (two per SM, each with half the threads); ampcg_tune_batched picks one.
constexpr int kBatchBlock = 1024;
constexpr int kBatchBlockSmall = 512;

// The staged SpMV in a block of BS / 32 warps: 3 stages per warp for
// binary32 values, 2 for binary64, so the stages of every variant fit in
// shared memory (two 512-thread blocks per SM fit as one 1024-thread block).
template <int UR> struct BatchStages { static constexpr int K = UR == P64 ? 2 : 3; };
template <int IT, int BS = kBatchBlock>
constexpr int batch_smem_bytes() {
  return staged_smem_bytes<P32, IT, 3>(BS / 32) > staged_smem_bytes<P64, IT, 2>(BS / 32)
             ? staged_smem_bytes<P32, IT, 3>(BS / 32)
             : staged_smem_bytes<P64, IT, 2>(BS / 32);
}
// Work partition over the block's threads.  Vectors that other threads of
// the block write during the launch are read with coherent loads
// (ld.global.ca, never the read-only path); __syncthreads orders the writes
// before the reads.
struct TeamPart {
  __device__ static __forceinline__ int64_t first() { return threadIdx.x; }
  __device__ static __forceinline__ int64_t count() { return blockDim.x; }
  __device__ static __forceinline__ int64_t warp() { return threadIdx.x >> 5; }
  __device__ static __forceinline__ int64_t warps() { return blockDim.x >> 5; }
  template <class T>
  __device__ static __forceinline__ T ldm(const T* p) { return __ldca(p); }
  template <int V, class T>
  __device__ static __forceinline__ void vldm(const T* p, T (&o)[V]) { vldca<V>(p, o); }
  template <int V, class T>
  __device__ static __forceinline__ void vldo(const T* p, T (&o)[V]) { vldca<V>(p, o); }
};

template <int UZ, int UR, int MT, int IT>
__device__ __forceinline__ void cta_iteration(const Sell& A, const Bufs& B, int64_t n, DevState* S,
                                              unsigned char* dsm, bool fused) {
  using Part = TeamPart;
  constexpr bool kSmall = (UR != P64) && (UZ != P64);
  // Alg. 3: scale, precondition, rho_k and beta (a second pass only when the
  // lagged scale made rho_k non-finite, reading R20); skipped when the
  // previous update step formed z_k and rho_k (fused: no scaling or the lagged
  // power of two, the same pair)
  for (int attempt = 0; attempt < 2 && !S->z_ready; ++attempt) {
    double rho = 0.0;
    Dot2 d2;
    precond_and_cast<UZ, UR, MT, 8, Part>(B, n, S, rho, d2);
    double v[1];
    if constexpr ((UR != P64) && (UZ != P64)) {
      v[0] = block_sum_dot2(d2, S->inv_sig);
    } else {
      v[0] = rho;
      block_sum_wide<1>(v);
    }
    if (threadIdx.x == 0) rho_step(S, v[0]);
    __syncthreads();
    if (!S->redo) break;
  }
  if (threadIdx.x == 0) S->phase_runs[2 * UZ + UR] += 1;
  __syncthreads();
  if (S->done) return;
  // Alg. 3: search direction (p_k is read by other threads' gathers)
  axpy_rows<UZ, 8, Part>(B, n, S);
  __syncthreads();
  // Alg. 3: q_k = A p_k, gamma_k, alpha_k
  {
    double gam = 0.0;
    Dot2 d2;
    if (A.maxw <= kStageW) spmv_rows_staged<UZ, UR, IT, Part, BatchStages<UR>::K>(A, B, S, gam, d2, dsm);
    else spmv_rows<UZ, UR, IT, Part>(A, B, S, gam, d2);
    double v[1];
    if constexpr ((UR != P64) && (UZ != P64)) {
      v[0] = block_sum_dot2(d2, 1.0);
    } else {
      v[0] = gam;
      block_sum_wide<1>(v);
    }
    if (threadIdx.x == 0) gamma_step(S, v[0]);
    __syncthreads();
    if (S->done) return;
  }
  // Alg. 3: x and r updates, delta_{k+1}, stopping test, next precisions;
  // fused: also z_{k+1} and rho_{k+1} in the same pass
  {
    double rr = 0.0, rho = 0.0;
    Dot2 d2, d2z;
    unsigned long long mx = 0ull;
    if (fused) {
      const PrecondScalars cn = PrecondScalars::next(S);
      update_precond_rows<UZ, UR, MT, 8, Part>(B, n, S, cn, rr, d2, mx, rho, d2z);
    } else {
      update_rows<UZ, UR, 8, Part>(B, n, S, rr, d2, mx);
    }
    double v[1], w[1] = {0.0};
    if constexpr (UR != P64) {
      v[0] = block_sum_dot2(d2, S->inv_sig2);
    } else {
      v[0] = rr;
      block_sum_wide<1>(v);
    }
    if (fused) {
      if constexpr (kSmall) {
        w[0] = block_sum_dot2(d2z, S->inv_sig);
      } else {
        w[0] = rho;
        block_sum_wide<1>(w);
      }
    }
    mx = block_max(mx);
    if (threadIdx.x == 0) {
      double d = update_step(S, v[0], mx);
      S->delta_hist[S->k] = d;
      if (fused && !S->done && S->uz == UZ && S->ur == UR) {
        rho_step(S, w[0]);
        S->z_ready = S->redo ? 0 : 1;
      }
    }
    __syncthreads();
  }
}

template <int MT, int IT>
__device__ __forceinline__ void cta_dispatch(int ph, const Sell& A, const Bufs& B, int64_t n, DevState* S,
                                             unsigned char* dsm, bool fused) {
  switch (ph) {
    case 0: cta_iteration<P64, P64, MT, IT>(A, B, n, S, dsm, fused); break;
    case 1: cta_iteration<P64, P32, MT, IT>(A, B, n, S, dsm, fused); break;
    case 2: cta_iteration<P32, P64, MT, IT>(A, B, n, S, dsm, fused); break;
    case 3: cta_iteration<P32, P32, MT, IT>(A, B, n, S, dsm, fused); break;
    case 4: cta_iteration<P16, P64, MT, IT>(A, B, n, S, dsm, fused); break;
    default: cta_iteration<P16, P32, MT, IT>(A, B, n, S, dsm, fused); break;
  }
}

template <int IT>
__device__ __forceinline__ void cta_dispatch_mt(int mt, int ph, const Sell& A, const Bufs& B, int64_t n,
                                                DevState* S, unsigned char* dsm, bool fused) {
  if (mt == M_JACOBI) cta_dispatch<M_JACOBI, IT>(ph, A, B, n, S, dsm, fused);
  else cta_dispatch<M_NONE, IT>(ph, A, B, n, S, dsm, fused);
}

// The whole solve of one system by one block (every thread calls it).
template <int IT>
__device__ void cta_solve(const BatchSys& D, DevState* S, int verify_refresh, unsigned char* dsm) {
  using Part = TeamPart;
  const Sell& A = D.A;
  const Bufs& B = D.B;
  const int64_t n = D.n;
  // the row loops use whole 8-element vectors: work in the context's padded buffers
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    D.bbuf[i] = D.b[i];
    B.x[i] = D.x[i];
  }
  __syncthreads();
  // Alg. 3: initial residual
  {
    double v[2] = {0.0, 0.0};
    unsigned long long mx = 0ull;
    init_rows<IT, Part>(A, B, v, mx);
    block_sum<2>(v);
    mx = block_max(mx);
    if (threadIdx.x == 0) S->delta_hist[0] = init_step(S, v[0], v[1], mx);
    __syncthreads();
  }
  int bodies = 0;
  const int limit = S->maxit + 1;
  // the update step forms z_{k+1}, rho_{k+1} where omega_{k+1} is known
  // before delta_{k+1} is reduced
  const bool fused = S->scale == SCALE_NONE || S->scale == SCALE_LINF_POW2_LAG;
  for (;;) {
    while (!S->done) {
      cta_dispatch_mt<IT>(D.mt, 2 * S->uz + S->ur, A, B, n, S, dsm, fused);
      if (++bodies > limit) {      // every iteration advances k or stops: cannot happen
        if (threadIdx.x == 0) {
          S->status = ST_INTERNAL;
          S->done = 1;
        }
        __syncthreads();
      }
    }
    // exit verification in FP64
    {
      double v[1] = {0.0};
      true_res_rows<IT, Part>(A, B, v);
      block_sum<1>(v);
      if (threadIdx.x == 0) S->true_relres = sqrt(v[0]) / S->nb;
      __syncthreads();
    }
    // reading R9
    const bool refresh = S->status == ST_OK && S->refreshes < verify_refresh && S->k < S->maxit &&
                         S->true_relres * S->nb > S->tol_nb;
    if (!refresh) break;
    double rr = 0.0;
    unsigned long long mx = 0ull;
    refresh_rows<Part>(B, n, S, rr, mx);
    double v[1] = {rr};
    block_sum<1>(v);
    mx = block_max(mx);
    if (threadIdx.x == 0) {
      int k = S->k;
      S->delta_hist[k] = refresh_step(S, v[0], mx);
    }
    __syncthreads();
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) D.x[i] = B.x[i];
}

// Persistent batched solver: blocks take systems order[next++] until the
// queue is empty.  tmpl: the initial state (policy, tol, maxit) shared by all
// systems.  Per system: x updated in place, the outcome in out[], histories
// in the system's arrays.
template <int IT, int BS>
__global__ void __launch_bounds__(BS, kBatchBlock / BS) k_batched(const BatchSys* sys, const int* order, int nsys,
                                                                  int* next, const DevState* tmpl,
                                                                  int verify_refresh, BatchOut* out) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ DevState S;
  __shared__ BatchSys D;   // the system's descriptor, shared by the block (not per-thread local memory)
  __shared__ int s_i;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_i = atomicAdd(next, 1);
    __syncthreads();
    const int q = s_i;
    if (q >= nsys) return;
    const int i = order[q];
    if (threadIdx.x == 0) D = sys[i];
    state_load(&S, tmpl);
    __syncthreads();
    if (threadIdx.x == 0) {
      S.delta_hist = D.delta_hist;
      S.prec_hist = D.prec_hist;
    }
    __syncthreads();
    cta_solve<IT>(D, &S, verify_refresh, dsm);
    __syncthreads();
    if (threadIdx.x == 0) {
      BatchOut o;
      o.iters = S.k;
      o.status = S.status;
      o.refreshes = S.refreshes;
      for (int j = 0; j < 3; ++j) o.switch_iter[j] = S.switch_iter[j];
      o.true_relres = S.true_relres;
      o.updated_relres = S.delta / S.nb;
      o.nb = S.nb;
      out[i] = o;
    }
  }
}

}  // namespace ampcg
