// device_util.cuh -- precision helpers and reductions for the AMP-PCG kernels.
//
// On B300 the FP64 pipe issues ~1.9 DFMA per clock per SM, and conversions
// to or from FP64 run at a similar rate, while the FP32/INT pipes issue ~108
// per clock.  The mixed-precision iteration therefore widens FP16/FP32 values
// to FP64 with integer operations (exact by construction) and rounds FP64 to
// FP16 with an integer implementation of IEEE round-to-nearest-even, so the
// only FP64-pipe instructions left are the FP64 arithmetic the method asks
// for (x update, FP64 residual/matrix products, inner-product accumulation).
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

namespace ampcg {

enum { P64 = 0, P32 = 1, P16 = 2 };

template <int P> struct Store;
template <> struct Store<P64> { using T = double; };
template <> struct Store<P32> { using T = float; };
template <> struct Store<P16> { using T = __half; };

// ---------------------------------------------------------------------------
// Exact widening to binary64 with integer operations only.

// f is +-0, a normal number, Inf or NaN (every binary16 value widened to
// binary32 is one of these).  Rebias the exponent (127 -> 1023) and move the
// 23 fraction bits to the top of the 52-bit fraction.
__device__ __forceinline__ double f2d_normal(float f) {
  unsigned u = __float_as_uint(f);
  unsigned s = u & 0x80000000u, a = u & 0x7fffffffu;
  unsigned hi = (a == 0u) ? s : (s | ((a >> 3) + (896u << 20)));
  if (a >= 0x7f800000u) hi = s | 0x7ff00000u | ((a >> 3) & 0x000fffffu);
  return __hiloint2double((int)hi, (int)(a << 29));
}

// Any binary32 value, integer operations only.  A subnormal a * 2^-149 with
// its leading one at bit p = 31 - clz(a) becomes 2^(p-149) (1 + fraction):
// the fraction is a shifted left by clz(a) - 8, the biased binary64 exponent
// is p - 149 + 1023 = 905 - clz(a).
__device__ __forceinline__ double f2d(float f) {
  unsigned u = __float_as_uint(f);
  unsigned s = u & 0x80000000u, a = u & 0x7fffffffu;
  unsigned hi = (a == 0u) ? s : (s | ((a >> 3) + (896u << 20)));
  unsigned lo = a << 29;
  if (a >= 0x7f800000u) hi = s | 0x7ff00000u | ((a >> 3) & 0x000fffffu);
  if (a != 0u && a < 0x00800000u) {
    int lz = __clz((int)a);
    unsigned m = (a << (lz - 8)) & 0x007fffffu;
    hi = s | ((unsigned)(905 - lz) << 20) | (m >> 3);
    lo = m << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float h2f(__half h) { return __half2float(h); }
__device__ __forceinline__ double h2d(__half h) { return f2d_normal(__half2float(h)); }

__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return f2d(v); }
__device__ __forceinline__ double to_f64(__half v) { return h2d(v); }

// ---------------------------------------------------------------------------
// Round-to-nearest-even of v * 2^sc into binary16.  Two steps: v * 2^sc is
// rounded to binary32 with round-to-odd (truncate the 52-bit fraction to 23
// bits and set the last bit when any discarded bit is set; 32-bit integer
// operations), then the hardware converts binary32 to binary16 with
// round-to-nearest-even.  Rounding to odd in a format with at least p + 2
// digits followed by round-to-nearest into p digits equals direct
// round-to-nearest (Boldo and Melquiond, "Emulation of FMA and correctly
// rounded sums: proved algorithms using rounding to odd", IEEE Trans.
// Computers 57, 2008); binary32 has 24 digits against binary16's 11.  Valid
// for |sc| < 900 (binary64 subnormal inputs lie far below binary16's range
// and give +-0).
__device__ __forceinline__ __half d2h_scaled(double v, int sc) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const unsigned s = hi & 0x80000000u;
  const int E = (int)((hi >> 20) & 0x7ffu);
  if (E == 0x7ff)
    return __ushort_as_half((unsigned short)((s >> 16) | (((hi & 0xfffffu) | lo) ? 0x7e00u : 0x7c00u)));
  if (E == 0) return __ushort_as_half((unsigned short)(s >> 16));
  const int e = E - 1023 + sc;                  // v * 2^sc = 1.f * 2^e
  if (e > 127) return __ushort_as_half((unsigned short)((s >> 16) | 0x7c00u));   // beyond binary32
  if (e < -150) return __ushort_as_half((unsigned short)(s >> 16));              // below binary16's
  const unsigned m23 = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned sticky = (lo & 0x1fffffffu) != 0u ? 1u : 0u;
  unsigned f;
  if (e >= -126) {
    f = s | ((unsigned)(e + 127) << 23) | m23 | sticky;
  } else {
    // binary32 subnormal: shift the significand (hidden bit included) right
    const int sh = -126 - e;                    // 1 .. 24
    const unsigned full = (1u << 23) | m23;
    const unsigned lost = (full & ((1u << sh) - 1u)) != 0u ? 1u : 0u;
    f = s | (full >> sh) | sticky | lost;
  }
  return __float2half_rn(__uint_as_float(f));
}

__device__ __forceinline__ __half d2h(double v) { return d2h_scaled(v, 0); }

// Rounding a binary64 value into precision P.
template <int P> __device__ __forceinline__ typename Store<P>::T round_from_f64(double v);
template <> __device__ __forceinline__ double round_from_f64<P64>(double v) { return v; }
template <> __device__ __forceinline__ float round_from_f64<P32>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ __half round_from_f64<P16>(double v) { return d2h(v); }

// Rounding a binary32 value into precision P (P64: exact widening).
template <int P> __device__ __forceinline__ typename Store<P>::T round_from_f32(float v);
template <> __device__ __forceinline__ double round_from_f32<P64>(float v) { return f2d(v); }
template <> __device__ __forceinline__ float round_from_f32<P32>(float v) { return v; }
template <> __device__ __forceinline__ __half round_from_f32<P16>(float v) { return __float2half_rn(v); }

// ---------------------------------------------------------------------------
// Vector access to V consecutive elements starting at an index that is a
// multiple of V (16-byte transactions when V elements fill whole 16-byte
// chunks).  Callers guarantee the V elements lie inside the allocation.
template <int V, class T>
__device__ __forceinline__ void vld(const T* __restrict__ p, T (&o)[V]) {
  if constexpr (V > 1 && (V * sizeof(T)) % 16 == 0) {
    constexpr int NQ = (int)(V * sizeof(T) / 16);
#pragma unroll
    for (int j = 0; j < NQ; ++j) reinterpret_cast<uint4*>(o)[j] = reinterpret_cast<const uint4*>(p)[j];
  } else {
#pragma unroll
    for (int j = 0; j < V; ++j) o[j] = p[j];
  }
}

// Read-only (non-coherent path) variant for arrays the kernel does not write.
template <int V, class T>
__device__ __forceinline__ void vldg(const T* __restrict__ p, T (&o)[V]) {
  if constexpr (V > 1 && (V * sizeof(T)) % 16 == 0) {
    constexpr int NQ = (int)(V * sizeof(T) / 16);
#pragma unroll
    for (int j = 0; j < NQ; ++j) reinterpret_cast<uint4*>(o)[j] = __ldg(reinterpret_cast<const uint4*>(p) + j);
  } else {
#pragma unroll
    for (int j = 0; j < V; ++j) o[j] = p[j];
  }
}

// Explicitly coherent variant (ld.global.ca, never the read-only path) for
// arrays other threads of the running kernel write between barriers.
template <int V, class T>
__device__ __forceinline__ void vldca(const T* p, T (&o)[V]) {
  if constexpr (V > 1 && (V * sizeof(T)) % 16 == 0) {
    constexpr int NQ = (int)(V * sizeof(T) / 16);
#pragma unroll
    for (int j = 0; j < NQ; ++j) reinterpret_cast<uint4*>(o)[j] = __ldca(reinterpret_cast<const uint4*>(p) + j);
  } else {
#pragma unroll
    for (int j = 0; j < V; ++j) o[j] = __ldca(p + j);
  }
}

// V elements through L2 only (data another block wrote in the same launch).
template <int V, class T>
__device__ __forceinline__ void vldcg(const T* __restrict__ p, T (&o)[V]) {
  if constexpr (V > 1 && (V * sizeof(T)) % 16 == 0) {
    constexpr int NQ = (int)(V * sizeof(T) / 16);
#pragma unroll
    for (int j = 0; j < NQ; ++j) reinterpret_cast<uint4*>(o)[j] = __ldcg(reinterpret_cast<const uint4*>(p) + j);
  } else {
#pragma unroll
    for (int j = 0; j < V; ++j) o[j] = __ldcg(p + j);
  }
}

// Accesses with an L2 evict-last hint (createpolicy; the policy is computed
// once and reused: the asm is not volatile).  The iteration vectors, re-read
// every iteration, are kept in L2 ahead of the streamed matrix.
__device__ __forceinline__ unsigned long long l2_policy_evict_last() {
  unsigned long long pol;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint4 ld16_keep(const void* p, unsigned long long pol) {
  uint4 v;
  asm volatile("ld.global.cg.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;\n"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void st16_keep(void* p, uint4 v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;\n" ::"l"(p), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w), "l"(pol)
               : "memory");
}
// scalar load through L2 with the hint; T of 2, 4 or 8 bytes
template <class T>
__device__ __forceinline__ T ld_keep(const T* p, unsigned long long pol) {
  if constexpr (sizeof(T) == 2) {
    unsigned short u;
    asm volatile("ld.global.cg.L2::cache_hint.u16 %0, [%1], %2;\n" : "=h"(u) : "l"(p), "l"(pol));
    return *reinterpret_cast<T*>(&u);
  } else if constexpr (sizeof(T) == 4) {
    unsigned u;
    asm volatile("ld.global.cg.L2::cache_hint.u32 %0, [%1], %2;\n" : "=r"(u) : "l"(p), "l"(pol));
    return *reinterpret_cast<T*>(&u);
  } else {
    unsigned long long u;
    asm volatile("ld.global.cg.L2::cache_hint.u64 %0, [%1], %2;\n" : "=l"(u) : "l"(p), "l"(pol));
    return *reinterpret_cast<T*>(&u);
  }
}
template <int V, class T>
__device__ __forceinline__ void vld_keep(const T* p, T (&o)[V], unsigned long long pol) {
  if constexpr ((V * sizeof(T)) % 16 == 0) {
    constexpr int NQ = (int)(V * sizeof(T) / 16);
#pragma unroll
    for (int j = 0; j < NQ; ++j)
      reinterpret_cast<uint4*>(o)[j] = ld16_keep(reinterpret_cast<const uint4*>(p) + j, pol);
  } else if constexpr (V * sizeof(T) == 8) {
    uint2 v;
    asm volatile("ld.global.cg.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;\n"
                 : "=r"(v.x), "=r"(v.y)
                 : "l"(p), "l"(pol));
    *reinterpret_cast<uint2*>(o) = v;
  } else {
#pragma unroll
    for (int j = 0; j < V; ++j) o[j] = __ldcg(p + j);
  }
}

// Stores the first m of V elements (all V with one vector store when m == V).
template <int V, class T>
__device__ __forceinline__ void vst(T* __restrict__ p, const T (&o)[V], int m) {
  if constexpr (V > 1 && (V * sizeof(T)) % 16 == 0) {
    if (m == V) {
      constexpr int NQ = (int)(V * sizeof(T) / 16);
#pragma unroll
      for (int j = 0; j < NQ; ++j) reinterpret_cast<uint4*>(p)[j] = reinterpret_cast<const uint4*>(o)[j];
      return;
    }
  } else if constexpr (V > 1 && V * sizeof(T) == 8) {
    if (m == V) {
      *reinterpret_cast<uint2*>(p) = *reinterpret_cast<const uint2*>(o);
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < V; ++j)
    if (j < m) p[j] = o[j];
}

// |v| as an order-preserving unsigned key (exact max-reduction).
__device__ __forceinline__ unsigned long long abs_key(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long abs_key(float v) {
  return (unsigned long long)__double_as_longlong(f2d(v)) & 0x7FFFFFFFFFFFFFFFull;
}

// ---------------------------------------------------------------------------
// Inner products accumulated to FP64-level accuracy.
//
// Binary64 operand: one FP64 fma per term, FP64 reductions.  Binary32/binary16
// operands: the product a*b is split exactly into h + l with an fma
// (two-product), h is added to a binary32 running sum with its rounding error
// captured exactly (two-sum), and the errors plus l are gathered in a binary32
// correction -- the compensated dot product Dot2 of Ogita, Rump and Oishi
// ("Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005).  A thread's
// (sum, correction) pair is reduced across its warp with the same two-sum
// step and converted to binary64 once per warp.  For a thread with n terms the
// error is at most about (n eps32)^2 times the sum of |terms| (n <= 32 here:
// <= 4e-12, typically ~1e-14), within the accuracy of a binary64 recursive sum
// of the same vector, while the work stays on B300's binary32 pipes (its
// binary64 pipe issues ~1/58 of the binary32 rate).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

struct Dot2 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    float h = __fmul_rn(a, b);
    float l = __fmaf_rn(a, b, -h);
    float t, e;
    two_sum(s, h, t, e);
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, l));
  }
  // warp reduction of the pairs (all lanes take part); lane 0 gets the total
  __device__ __forceinline__ void warp_reduce() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float s2 = __shfl_down_sync(0xffffffffu, s, o);
      float c2 = __shfl_down_sync(0xffffffffu, c, o);
      float t, e;
      two_sum(s, s2, t, e);
      s = t;
      c = __fadd_rn(__fadd_rn(c, c2), e);
    }
  }
  __device__ __forceinline__ double to_f64() const { return __dadd_rn(f2d(s), f2d(c)); }
};

// ---------------------------------------------------------------------------
// Reductions.  Fixed shapes, so results are reproducible run to run.

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long warp_max(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_down_sync(0xffffffffu, v, o);
    v = (w > v) ? w : v;
  }
  return v;
}

// Sum of NV values per block; result valid in thread 0.  blockDim.x must be
// a multiple of 32 and at most 1024.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) v[j] = warp_sum(v[j]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) sh[j][wid] = v[j];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double t = (lane < nw) ? sh[j][lane] : 0.0;
      v[j] = warp_sum(t);
    }
  }
}

// block_sum for blocks of 1024 threads (blockDim.x a multiple of 256, at most
// 1024).  The values go through shared memory: thread r < 256 adds values
// r, r + 256, ... in that order, each of those 8 warps reduces by a shuffle
// tree, and warp 0 adds the 8 warp totals with 3 more levels.  At 1024
// threads it issues 67 FP64 warp-instructions per value against 165 for a
// shuffle tree in every warp, which matters on B300, whose FP64 pipe takes
// 16 cycles per warp-instruction.
template <int NV>
__device__ __forceinline__ void block_sum_wide(double (&v)[NV]) {
  __shared__ double sh[NV][1024];
  __shared__ double sw[NV][8];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) sh[j][t] = v[j];
  __syncthreads();
  if (t < 256) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double a = sh[j][t];
      for (int u = t + 256; u < (int)blockDim.x; u += 256) a += sh[j][u];
      a = warp_sum(a);
      if (lane == 0) sw[j][wid] = a;
    }
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double a = lane < 8 ? sw[j][lane] : 0.0;
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
      v[j] = a;
    }
  }
}

// Block total of per-thread Dot2 pairs, scaled by `scale` (a power of two);
// valid in thread 0.  Binary64 work: one add per warp plus warp 0's tree.
__device__ __forceinline__ double block_sum_dot2(Dot2 d, double scale) {
  __shared__ double shd[32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  d.warp_reduce();
  __syncthreads();
  if (lane == 0) shd[wid] = __dmul_rn(d.to_f64(), scale);
  __syncthreads();
  double t = 0.0;
  if (wid == 0) t = warp_sum(lane < nw ? shd[lane] : 0.0);
  return t;
}

__device__ __forceinline__ unsigned long long block_max(unsigned long long v) {
  __shared__ unsigned long long shm[32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) shm[wid] = v;
  __syncthreads();
  if (wid == 0) v = warp_max(lane < nw ? shm[lane] : 0ull);
  return v;
}

// block_sum_dot2 of NS pairs (scaled by scale[k]) and block_max in one pass:
// the same per-warp reductions and the same fixed-order totals as the
// separate calls, hence the same bits, with two block barriers instead of
// 2 (NS + 1).  Totals valid in warp 0 (thread 0 uses them).
template <int NS>
__device__ __forceinline__ void block_sums_dot2_max(Dot2 (&d)[NS], const double (&scale)[NS], double (&out)[NS],
                                                    unsigned long long& mx) {
  __shared__ double shd[NS][32];
  __shared__ unsigned long long shm[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NS; ++k) d[k].warp_reduce();
  mx = warp_max(mx);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NS; ++k) shd[k][wid] = __dmul_rn(d[k].to_f64(), scale[k]);
    shm[wid] = mx;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NS; ++k) out[k] = warp_sum(lane < nw ? shd[k][lane] : 0.0);
    mx = warp_max(lane < nw ? shm[lane] : 0ull);
  }
}

// block_sum_wide of NV values and block_max in one pass (the same sums and
// bits as the separate calls; two block barriers instead of four).
template <int NV>
__device__ __forceinline__ void block_sum_wide_max(double (&v)[NV], unsigned long long& mx) {
  __shared__ double sh[NV][1024];
  __shared__ double sw[NV][8];
  __shared__ unsigned long long shm[32];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) sh[j][t] = v[j];
  mx = warp_max(mx);
  if (lane == 0) shm[wid] = mx;
  __syncthreads();
  if (t < 256) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double a = sh[j][t];
      for (int u = t + 256; u < (int)blockDim.x; u += 256) a += sh[j][u];
      a = warp_sum(a);
      if (lane == 0) sw[j][wid] = a;
    }
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double a = lane < 8 ? sw[j][lane] : 0.0;
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
      v[j] = a;
    }
    mx = warp_max(lane < nw ? shm[lane] : 0ull);
  }
}

// Single-pass grid reduction: every block publishes its partials, then takes
// a ticket; the block that draws the last ticket sees all partials.  Returns
// true in every thread of that block.  The last block must reset *ticket.
__device__ __forceinline__ bool last_block(unsigned int* ticket) {
  __shared__ bool is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// Grid barrier of a cooperative launch (every block resident), optionally
// with a grid-wide sum (MODE 1) or sum and max (MODE 2) of one partial per
// block.  Every block publishes its partials, then takes a ticket (fence,
// atomic add; the counter only grows: the tickets of one barrier take it from
// a multiple of gridDim.x to the next one) and kPollers of its warps poll the
// counter until it reaches that multiple (measured on B300: about 1.45 us
// per barrier with one poller, against about 2.05 us when the last block
// writes a separate release word; staggered pollers shave a further ~0.2 us
// off each barrier of the iteration kernel).  Then
// warp 0 of every block sums the partials in the same fixed order (each lane
// a strided run, loads issued eight at a time, then a fixed tree), so all
// blocks hold the same totals: one warp per block keeps the FP64 work small
// (B300's FP64 pipe issues 1/58 of the FP32 rate).
// All launches that share a barrier use the same grid, and the host zeroes
// it before each solve.  A wait that runs out after kBarrierSpin polls (about
// a second; it cannot happen with every block resident) returns false in
// every thread of the block instead of hanging.  The partials alternate
// between two halves of part and of pmax (gridDim.x entries each for the
// single-sum forms; the two-sum form has its own halves after them),
// selected by the launch's barrier count `nb`: a block that has passed
// barrier j may publish for barrier j + 1 while another still reads barrier
// j's partials.
struct GridSumBarrier {
  unsigned long long arrive;   // tickets taken
  unsigned long long pad[3];
};
constexpr long long kBarrierSpin = 1ll << 21;
constexpr int kPollers = 4;   // warps of a block polling a grid barrier (blocks of >= 128 threads)

template <int NSUM, bool MAX>
__device__ __forceinline__ bool grid_barrier_sums(GridSumBarrier* g, double* part, unsigned long long* pmax,
                                                  int& nb, const double* v, unsigned long long mx, double* tot,
                                                  unsigned long long& mtot, long long spin);
template <int MODE>
__device__ __forceinline__ bool grid_reduce_barrier(GridSumBarrier* g, double* part, unsigned long long* pmax,
                                                    int& nb, double v, unsigned long long mx, double& tot,
                                                    unsigned long long& mtot, long long spin = kBarrierSpin);

// Fixed-order sum of G partials (block g's value j at part[g*stride + j]) in
// the last block; thread 0 gets the totals.  Thread t adds partials t, t + B,
// t + 2B, ... in that order; the loads of up to four of them are issued
// before the first add, so the tail pays one memory round trip, not G / B.
template <int NV>
__device__ __forceinline__ void final_sum(const double* part, int G, int stride, double (&out)[NV]) {
#pragma unroll
  for (int j = 0; j < NV; ++j) out[j] = 0.0;
  const int B = blockDim.x;
  for (int g0 = threadIdx.x; g0 < G; g0 += 4 * B) {
    double v[4][NV];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int g = g0 + u * B;
#pragma unroll
      for (int j = 0; j < NV; ++j) v[u][j] = (g < G) ? __ldcg(part + (size_t)g * stride + j) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (g0 + u * B < G) {
#pragma unroll
        for (int j = 0; j < NV; ++j) out[j] += v[u][j];
      }
    }
  }
  block_sum<NV>(out);
}

__device__ __forceinline__ unsigned long long final_max(const unsigned long long* part, int G) {
  unsigned long long m = 0ull;
  const int B = blockDim.x;
  for (int g0 = threadIdx.x; g0 < G; g0 += 4 * B) {
    unsigned long long v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = (g0 + u * B < G) ? __ldcg(part + g0 + u * B) : 0ull;
#pragma unroll
    for (int u = 0; u < 4; ++u) m = v[u] > m ? v[u] : m;
  }
  return block_max(m);
}

// final_sum<NV> and final_max together: all loads issued before any use.
template <int NV>
__device__ __forceinline__ unsigned long long final_sum_max(const double* part, int stride,
                                                            const unsigned long long* pmax, int G,
                                                            double (&out)[NV]) {
#pragma unroll
  for (int j = 0; j < NV; ++j) out[j] = 0.0;
  unsigned long long m = 0ull;
  const int B = blockDim.x;
  for (int g0 = threadIdx.x; g0 < G; g0 += 4 * B) {
    double v[4][NV];
    unsigned long long w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int g = g0 + u * B;
#pragma unroll
      for (int j = 0; j < NV; ++j) v[u][j] = (g < G) ? __ldcg(part + (size_t)g * stride + j) : 0.0;
      w[u] = (g < G) ? __ldcg(pmax + g) : 0ull;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (g0 + u * B < G) {
#pragma unroll
        for (int j = 0; j < NV; ++j) out[j] += v[u][j];
      }
      m = w[u] > m ? w[u] : m;
    }
  }
  block_sum<NV>(out);
  return block_max(m);
}

// Grid barrier with NSUM grid-wide sums (0, 1 or 2 per block, v[j] valid in
// thread 0; block g's partial j at part[2G + parity * 2G + g * NSUM + j],
// parity = the barrier's count in the launch mod 2; part holds 6G doubles)
// and, with
// MAX, the grid-wide maximum of the blocks' mx; tot[j] and mtot end up in
// every thread.  spin: polls per polling warp before the wait gives up.  The
// block passes the barrier when any of its pollers saw it complete; it fails
// only when every poller ran out.
template <int NSUM, bool MAX>
__device__ __forceinline__ bool grid_barrier_sums(GridSumBarrier* g, double* part, unsigned long long* pmax,
                                                  int& nb, const double* v, unsigned long long mx, double* tot,
                                                  unsigned long long& mtot, long long spin) {
  static_assert(NSUM >= 0 && NSUM <= 2, "0, 1 or 2 sums");
  __shared__ double s_tot[2];
  __shared__ unsigned long long s_max;
  // its partials live after the single-sum forms' two halves (2G doubles):
  // halves of 2G doubles at 2G and 4G, so consecutive barriers of either kind
  // never share entries
  const int parity = nb++ & 1;
  if constexpr (NSUM >= 1) part += 2 * (int)gridDim.x + parity * 2 * (int)gridDim.x;
  if constexpr (MAX) pmax += parity * (int)gridDim.x;
  __shared__ unsigned long long s_target;
  __shared__ volatile int s_seen;
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NSUM; ++j) part[blockIdx.x * NSUM + j] = v[j];
    if constexpr (MAX) pmax[blockIdx.x] = mx;
    __threadfence();
    const unsigned long long G = gridDim.x;
    const unsigned long long a = atomicAdd(&g->arrive, 1ull);
    s_target = (a / G + 1) * G;
    s_seen = 0;
  }
  __syncthreads();
  // kPollers warps poll, started a quarter of a round trip apart, so that the
  // completion is seen about a quarter round trip after it lands instead of
  // half a round trip on average; the first to see it tells the others
  if ((threadIdx.x & 31) == 0 && (threadIdx.x >> 5) < kPollers) {
    const int w = threadIdx.x >> 5;
    if (w) __nanosleep(150u * (unsigned)w);
    const unsigned long long target = s_target;
    for (long long it = 0;; ++it) {
      if (s_seen) break;
      unsigned long long r;
      asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(r) : "l"(&g->arrive) : "memory");
      if (r >= target) {
        s_seen = 1;
        break;
      }
      if (it >= spin) break;
    }
    __threadfence();
  }
  __syncthreads();
  const bool ok = s_seen != 0;
  if (!ok) return false;   // uniform across the block: s_seen is read after the barrier
  if constexpr (NSUM >= 1 || MAX) {
    // warp q < NSUM sums partial q, warp NSUM takes the max: each lane adds
    // partials lane, lane + 32, ... in that order (loads of five issued
    // before the first add: one memory round trip up to 160 blocks), then a
    // fixed tree
    constexpr int U = 5;
    const int wq = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int G = gridDim.x;
    if (wq < NSUM) {
      double t = 0.0;
      for (int i0 = lane; i0 < G; i0 += 32 * U) {
        double pv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int i = i0 + 32 * u;
          pv[u] = i < G ? __ldcg(part + (size_t)i * NSUM + wq) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (i0 + 32 * u < G) t += pv[u];
      }
      t = warp_sum(t);
      if (lane == 0) s_tot[wq] = t;
    } else if (MAX && wq == NSUM) {
      unsigned long long m = 0ull;
      for (int i0 = lane; i0 < G; i0 += 32 * U) {
        unsigned long long pw[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int i = i0 + 32 * u;
          pw[u] = i < G ? __ldcg(pmax + i) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) m = pw[u] > m ? pw[u] : m;
      }
      m = warp_max(m);
      if (lane == 0) s_max = m;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NSUM; ++j) tot[j] = s_tot[j];
    if constexpr (MAX) mtot = s_max;
  }
  return true;
}

// The single-sum forms: MODE 0 plain barrier, 1 one sum, 2 one sum and the
// max; block g's partial at part[parity * G + g] (halves G apart).  Kept
// apart from grid_barrier_sums (measured on B300: the shared two-sum code
// cost 0.6-2.5 us per iteration of the persistent kernel in these forms).
template <int MODE>
__device__ __forceinline__ bool grid_reduce_barrier(GridSumBarrier* g, double* part, unsigned long long* pmax,
                                                    int& nb, double v, unsigned long long mx, double& tot,
                                                    unsigned long long& mtot, long long spin) {
  __shared__ double s_tot;
  __shared__ unsigned long long s_max;
  const int half = (nb++ & 1) * (int)gridDim.x;
  if constexpr (MODE >= 1) part += half;
  if constexpr (MODE == 2) pmax += half;
  __shared__ unsigned long long s_target;
  __shared__ volatile int s_seen;
  __syncthreads();
  if (threadIdx.x == 0) {
    if constexpr (MODE >= 1) part[blockIdx.x] = v;
    if constexpr (MODE == 2) pmax[blockIdx.x] = mx;
    __threadfence();
    const unsigned long long G = gridDim.x;
    const unsigned long long a = atomicAdd(&g->arrive, 1ull);
    s_target = (a / G + 1) * G;
    s_seen = 0;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0 && (threadIdx.x >> 5) < kPollers) {
    const int w = threadIdx.x >> 5;
    if (w) __nanosleep(150u * (unsigned)w);
    const unsigned long long target = s_target;
    for (long long it = 0;; ++it) {
      if (s_seen) break;
      unsigned long long r;
      asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(r) : "l"(&g->arrive) : "memory");
      if (r >= target) {
        s_seen = 1;
        break;
      }
      if (it >= spin) break;
    }
    __threadfence();
  }
  __syncthreads();
  if constexpr (MODE >= 1) {
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      const int G = gridDim.x;
      double t = 0.0;
      unsigned long long m = 0ull;
      for (int i0 = lane; i0 < G; i0 += 32 * 8) {
        double pv[8];
        unsigned long long pw[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = i0 + 32 * u;
          pv[u] = i < G ? __ldcg(part + i) : 0.0;
          if constexpr (MODE == 2) pw[u] = i < G ? __ldcg(pmax + i) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (i0 + 32 * u < G) t += pv[u];
          if constexpr (MODE == 2) m = pw[u] > m ? pw[u] : m;
        }
      }
      t = warp_sum(t);
      if constexpr (MODE == 2) m = warp_max(m);
      if (lane == 0) {
        s_tot = t;
        s_max = m;
      }
    }
    __syncthreads();
    tot = s_tot;
    if constexpr (MODE == 2) mtot = s_max;
  }
  return s_seen != 0;   // passed when any poller saw the barrier complete
}

}  // namespace ampcg
