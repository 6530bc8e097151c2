// bsr.cuh -- block-row kernels for matrices given as block CSR with 3 x 3
// blocks (ampcg_create_bsr with bs = 3, e.g. vector-valued elasticity).
//
// The scalar sliced layout stores every entry with its own column offset and
// a row gathers each of its ~81 operands itself.  Here one thread owns a
// block row (its 3 scalar rows): per stored block it reads one block column
// index and the block's 9 values, gathers the 3 operands x[3J..3J+2] once and
// uses them for all 3 rows -- a third of the index traffic and of the
// gathers.  Each scalar row's products are accumulated in the same order as
// in the scalar kernels (blocks by ascending block column, then the 3 columns
// of the block), one fma per entry, so the results are bitwise those of the
// scalar path (and of the oracle on the expanded matrix).
//
// Layout: block rows in slices of 32 (one per lane of a warp); block j of the
// slice's lane-th block row has its block column at bcol[boff[s] + 32 j +
// lane] and its 9 values (row-major, v = 3 i + c) at
// val[9 (boff[s] + 32 j) + 32 v + lane], so each of a block's 9 values is one
// coalesced load across the warp.  Block rows shorter than the slice are
// padded with zero blocks on their own block column.  The block layout is
// derived from the scalar sliced layout (which holds the same values in CSR
// order for rows this wide), so it follows every value update.
#pragma once
#include "kernels.cuh"

namespace ampcg {

struct BSell {
  int64_t nb, nbs;         // block rows, slices of 32 block rows
  const long long* boff;   // [nbs] first block of the slice
  const int* bw;           // [nbs] slice width in blocks
  const int* bcol;         // [32 sum bw] block columns
  const double* v64;       // [9 * 32 sum bw] values, FP64
  const float* v32;        //                 FP32
  const double* ah64;      // Chebyshev: D^-1/2 A D^-1/2 in FP64, FP32, FP16 (else null)
  const float* ah32;
  const __half* ah16;
};

template <int P> __device__ __forceinline__ const typename Store<P>::T* bvals(const BSell& A);
template <> __device__ __forceinline__ const double* bvals<P64>(const BSell& A) { return A.v64; }
template <> __device__ __forceinline__ const float* bvals<P32>(const BSell& A) { return A.v32; }
template <int P> __device__ __forceinline__ const typename Store<P>::T* bahat(const BSell& A);
template <> __device__ __forceinline__ const double* bahat<P64>(const BSell& A) { return A.ah64; }
template <> __device__ __forceinline__ const float* bahat<P32>(const BSell& A) { return A.ah32; }
template <> __device__ __forceinline__ const __half* bahat<P16>(const BSell& A) { return A.ah16; }

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// acc[i] = fma chain over the block row's entries of row i: values va (type
// TA, widened to the accumulator by cva), operands x (type TX, widened by
// cvx), accumulator type TACC.  The next block's index and values are loaded
// before the current block's gathers.
template <class TACC, class TA, class TX, class CvA, class CvX>
__device__ __forceinline__ void block_row_sum(const BSell& A, const TA* __restrict__ va, long long base9,
                                              long long bbase, int w, const TX* __restrict__ x,
                                              TACC (&acc)[3], CvA cva, CvX cvx) {
#pragma unroll
  for (int i = 0; i < 3; ++i) acc[i] = TACC(0);
  if (w <= 0) return;
  int J = __ldg(A.bcol + bbase);
  TA a[9];
#pragma unroll
  for (int v = 0; v < 9; ++v) a[v] = __ldg(va + base9 + 32 * v);
  for (int j = 0; j < w; ++j) {
    int Jn = J;
    TA an[9];
    if (j + 1 < w) {
      Jn = __ldg(A.bcol + bbase + 32 * (j + 1));
#pragma unroll
      for (int v = 0; v < 9; ++v) an[v] = __ldg(va + base9 + 288 * (j + 1) + 32 * v);
    }
    const TX x0 = x[3 * (int64_t)J], x1 = x[3 * (int64_t)J + 1], x2 = x[3 * (int64_t)J + 2];
    const TACC g0 = cvx(x0), g1 = cvx(x1), g2 = cvx(x2);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      acc[i] = fma_t(cva(a[3 * i]), g0, acc[i]);
      acc[i] = fma_t(cva(a[3 * i + 1]), g1, acc[i]);
      acc[i] = fma_t(cva(a[3 * i + 2]), g2, acc[i]);
    }
    if (j + 1 < w) {
      J = Jn;
#pragma unroll
      for (int v = 0; v < 9; ++v) a[v] = an[v];
    }
  }
}

// Alg. 3 matrix product q = A p in u_r with A's copy in u_r (block layout),
// gamma = q^T p, alpha: the block-row counterpart of k_spmv (wide rows).
template <int UZ, int UR>
__global__ void __launch_bounds__(256) k_bspmv(BSell A, Bufs B, DevState* st) {
  using TZ = typename Store<UZ>::T;
  using TR = typename Store<UR>::T;
  constexpr bool kSmall = (UR != P64) && (UZ != P64);
  __shared__ DevState S;
  if (!state_enter(&S, st, UZ, UR)) return;
  const TZ* __restrict__ p = (const TZ*)(S.pcur ? B.p[0] : B.p[1]);
  TR* __restrict__ q = (TR*)B.q;
  const TR* __restrict__ va = bvals<UR>(A);
  double gam = 0.0;
  Dot2 d2;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = warp; s < A.nbs; s += nwarps) {
    const int64_t I = s * 32 + lane;
    if (I >= A.nb) continue;
    const long long b0 = __ldg(A.boff + s);
    const int w = __ldg(A.bw + s);
    TR acc[3];
    block_row_sum<TR>(A, va, 9 * b0 + lane, b0 + lane, w, p, acc, [](TR a) { return a; },
                      [](TZ v) { return PToR<UZ, UR>::cv(v); });
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int64_t row = 3 * I + i;
      q[row] = acc[i];
      const TZ pr = p[row];
      if constexpr (kSmall) d2.add((float)acc[i], (float)pr);
      else gam = fma(to_f64(acc[i]), to_f64(pr), gam);
    }
  }
  double v[1];
  if constexpr (kSmall) {
    v[0] = block_sum_dot2(d2, 1.0);
  } else {
    v[0] = gam;
    block_sum<1>(v);
  }
  if (threadIdx.x == 0) B.part[blockIdx.x] = v[0];
  if (!last_block(&st->ticket[1])) return;
  state_load(&S, st);
  double tot[1];
  final_sum<1>(B.part, gridDim.x, 1, tot);
  if (threadIdx.x == 0) {
    S.ticket[1] = 0u;
    gamma_step(&S, tot[0]);
  }
  state_store(st, &S);
}

// One Chebyshev step j >= 1 (reading R8) with the block layout of Ahat in u_z:
// t = Ahat d_{j-1} (accumulated as k_cheb_step does: FP64 for u_z = FP64,
// else FP32, then rounded to u_z), res -= t, d_j = c1 d_{j-1} + c2 res,
// u += d_j -- the same operations as k_cheb_step, 3 rows per thread.
template <int UZ, int UR>
__global__ void __launch_bounds__(256) k_bcheb_step(BSell A, Cheb C, DevState* st, int j, double c1, double c2) {
  using TZ = typename Store<UZ>::T;
  {
    const int dn = st->done, uz = st->uz, ur = st->ur;
    if (dn || uz != UZ || ur != UR) return;
  }
  const TZ* __restrict__ dp = (const TZ*)(((j - 1) & 1) ? C.d[1] : C.d[0]);
  TZ* dn = (TZ*)((j & 1) ? C.d[1] : C.d[0]);
  TZ* res = (TZ*)C.res;
  TZ* u = (TZ*)C.u;
  const float c1f = __double2float_rn(c1), c2f = __double2float_rn(c2);
  const TZ* __restrict__ va = bahat<UZ>(A);
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = warp; s < A.nbs; s += nwarps) {
    const int64_t I = s * 32 + lane;
    if (I >= A.nb) continue;
    const long long b0 = __ldg(A.boff + s);
    const int w = __ldg(A.bw + s);
    TZ t[3];
    if constexpr (UZ == P64) {
      double acc[3];
      block_row_sum<double>(A, va, 9 * b0 + lane, b0 + lane, w, dp, acc, [](double a) { return a; },
                            [](double v) { return v; });
#pragma unroll
      for (int i = 0; i < 3; ++i) t[i] = acc[i];
    } else if constexpr (UZ == P32) {
      float acc[3];
      block_row_sum<float>(A, va, 9 * b0 + lane, b0 + lane, w, dp, acc, [](float a) { return a; },
                           [](float v) { return v; });
#pragma unroll
      for (int i = 0; i < 3; ++i) t[i] = acc[i];
    } else {
      float acc[3];
      block_row_sum<float>(A, va, 9 * b0 + lane, b0 + lane, w, dp, acc, [](__half a) { return __half2float(a); },
                           [](__half v) { return __half2float(v); });
#pragma unroll
      for (int i = 0; i < 3; ++i) t[i] = __float2half_rn(acc[i]);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int64_t row = 3 * I + i;
      TZ rs = sub_u<UZ>(res[row], t[i]);
      TZ dd;
      if constexpr (UZ == P64) dd = fma(c1, dp[row], __dmul_rn(c2, rs));
      else if constexpr (UZ == P32) dd = __fmaf_rn(c1f, dp[row], __fmul_rn(c2f, rs));
      else dd = __float2half_rn(__fmaf_rn(c1f, __half2float(dp[row]), __fmul_rn(c2f, __half2float(rs))));
      res[row] = rs;
      dn[row] = dd;
      u[row] = add_u<UZ>(u[row], dd);
    }
  }
}

// q = A p on caller arrays with the block layout (FP64 or FP32 values,
// accumulated in that precision), for parity tests of the block kernels.
template <int UR>
__global__ void __launch_bounds__(256) k_bspmv_step(BSell A, const void* p, void* q) {
  using TR = typename Store<UR>::T;
  const TR* __restrict__ pp = (const TR*)p;
  TR* __restrict__ qq = (TR*)q;
  const TR* __restrict__ va = bvals<UR>(A);
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = warp; s < A.nbs; s += nwarps) {
    const int64_t I = s * 32 + lane;
    if (I >= A.nb) continue;
    const long long b0 = __ldg(A.boff + s);
    const int w = __ldg(A.bw + s);
    TR acc[3];
    block_row_sum<TR>(A, va, 9 * b0 + lane, b0 + lane, w, pp, acc, [](TR a) { return a; }, [](TR v) { return v; });
#pragma unroll
    for (int i = 0; i < 3; ++i) qq[3 * I + i] = acc[i];
  }
}

#ifndef AMPCG_INSTANTIATION_UNIT
// Slice widths in blocks: rows 3I of the slice hold 3 entries per block.
__global__ void k_bslice_width(int64_t nb, int64_t nbs, const int* rowptr, int* bw) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nbs) return;
  int w = 0;
  for (int l = 0; l < 32; ++l) {
    const int64_t I = s * 32 + l;
    if (I < nb) {
      const int len = (rowptr[3 * I + 1] - rowptr[3 * I]) / 3;
      w = len > w ? len : w;
    }
  }
  bw[s] = w;
}

// Fills the block layout (block columns, values in two precisions, and the
// Chebyshev Ahat copies when given) from the scalar sliced layout, in which
// entry e = 3 k + c of row 3 I + i (e < the row's CSR length) is column c of
// the row's k-th block.  One thread per block row.
template <int IT>
__global__ void k_bfill(Sell S, const int* rowptr, BSell B, int* bcol, double* v64, float* v32,
                        const double* sah64, double* ah64, float* ah32, __half* ah16) {
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t s = I >> 5;
  const int lane = (int)(I & 31);
  if (s >= B.nbs) return;
  const long long b0 = B.boff[s];
  const int w = B.bw[s];
  const int nblk = I < B.nb ? (rowptr[3 * I + 1] - rowptr[3 * I]) / 3 : 0;
  for (int k = 0; k < w; ++k) {
    const long long bi = b0 + 32ll * k + lane;
    int J = (int)(I < B.nb ? I : 0);
    if (k < nblk) {
      const int r0 = (int)(3 * I);
      const long long e0 = S.off[r0 >> 5] + (r0 & 31) + 32ll * (3 * k);
      J = col_at<IT>(S, e0, r0) / 3;
    }
    bcol[bi] = J;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double v = 0.0, ah = 0.0;
        if (k < nblk) {
          const int r = (int)(3 * I + i);
          const long long e = S.off[r >> 5] + (r & 31) + 32ll * (3 * k + c);
          v = S.v64[e];
          if (sah64) ah = sah64[e];
        }
        const long long q = 9ll * (b0 + 32ll * k) + 32 * (3 * i + c) + lane;
        v64[q] = v;
        v32[q] = __double2float_rn(v);
        if (ah64) {
          ah64[q] = ah;
          ah32[q] = __double2float_rn(ah);
          ah16[q] = d2h(ah);
        }
      }
    }
  }
}
#endif

}  // namespace ampcg
