// kernels.cuh -- AMP-PCG (Algorithm 3 of Guo, de Sturler, Warburton) on one
// B300.  The row loops of each step of Alg. 3 are device functions shared by
// three kernel families:
//   k_loop (Jacobi or no preconditioner, slices at most kStageW wide): the
//     iteration loop of one precision pair in one cooperative launch; grid
//     barriers (with the grid sums) separate the steps.
//   the kernel sequence (Chebyshev preconditioner, wide slices): the
//     precondition step (k_precond_dir, or the Chebyshev kernels then k_axpy),
//     k_spmv and k_update; each grid reduction is single-pass (last-block
//     ticket) and its last block runs the scalar step of the algorithm.
//   k_batched (batched.cuh): one block per system.
// The launch-by-launch mode (per-kernel timing) runs the same kernels, k_loop
// one iteration per launch.
// The steps: scaling and preconditioning y = omega r (u_r), z = M^-1 y (u_z),
// rho and beta; search direction p = z + beta p (u_z); q = A p (u_r), gamma
// and alpha; x += alpha p (FP64), r -= alpha q (u_r), ||r||, max|r|, the
// stopping test, indicator and selector for the next iteration, omega.  No
// host synchronisation happens inside the loop.  Each kernel is specialised
// for one precision pair (u_z, u_r) (phase index 2 u_z + u_r), so every
// variant gets its own register allocation; the pair of an iteration is
// decided on the device and selects the variant through a conditional SWITCH
// node of the loop graph (or through the host, in the launch-by-launch mode).
#pragma once
#include <type_traits>
#include "device_util.cuh"

namespace ampcg {

enum { CRIT_WINDOW = 0, CRIT_LINEAR = 1, CRIT_FIXED = 2 };
enum { SCALE_NONE = 0, SCALE_L2 = 1, SCALE_LINF_POW2 = 2, SCALE_LINF_POW2_LAG = 3 };
enum { M_NONE = 0, M_JACOBI = 1, M_CHEBYSHEV = 2 };
// ST_TIMEOUT: a bounded grid-barrier wait ran out (every block of a cooperative
// launch is resident, so this means a block never arrived)
enum { ST_OK = 0, ST_NOT_CONVERGED = 1, ST_BREAKDOWN = -3, ST_NONFINITE = -4, ST_INTERNAL = -5,
       ST_TIMEOUT = -7 };

// Switch value for an iteration that must not run (solve finished): matches
// no body of the SWITCH node, so nothing is launched.
#define AMPCG_PHASE_NONE 6



// Unit roundoff of binary32 (2^-24), the eps_32 of Eq. (eta_k).
#define AMPCG_EPS32 5.9604644775390625e-08

// The last kRing residual norms delta_t live in the state itself (dring[t %
// kRing]), so the selector's indicator window arrives with the one
// cooperative load of the state in a reduction tail (d <= kRing - 2,
// ell <= kRing - 1).
constexpr int kRing = 64;

struct __align__(16) DevState {
  // iteration control
  int k, done, status, maxit;
  int uz, ur;          // precisions of the current iteration
  int uz_p;            // precision p_{k-1} is stored in
  int r_cast, p_cast;  // storage conversions due at this iteration
  int pcur;            // p_{k-1} lives in pbuf[pcur]
  int first;           // no search direction yet
  int refreshes;
  int switch_iter[3];
  int k_body;          // iteration counter seen by the previous outer-loop body end
  int k_chunk;         // iteration counter seen by the previous inner-loop chunk end
  int loop_runs;       // outer-loop bodies run (launch accounting)
  int chunk_runs[6];   // inner-loop chunks run per pair 2 u_z + u_r
  // policy
  int criterion, u0, d, ell, scale, latch, fixed_uz, fixed_ur;
  double C, tau_zs, tau_zh, tol;
  // scalars (FP64, Sec. 4: all scalar work in double precision)
  double nb, tol_nb, delta, maxr, omega;
  int omega_pow2, omega_e;  // omega = 2^omega_e when omega_pow2
  float omega_f, beta_f, alpha_f;
  float sig_f;              // 2^sig_e: exact scale of r in binary32 dot products
  int sig_e;
  double inv_sig, inv_sig2; // 2^-sig_e, 2^-2 sig_e
  // selector brackets (prep_selector)
  double inv_tol_nb, tzs_lo, tzs_hi, tzh_lo, tzh_hi, c_lin;
  double rho, rho_prev, beta, gamma, alpha, true_relres;
  double maxr_prev;          // max|r_{k-1}| (lagged scale, reading R20)
  int z_ready;               // z_k and rho_k already formed (by the previous update step)
  int omega_exact;           // omega_k retried with max|r_k| (reading R20)
  int redo;                  // set by the scalar step: form y_k, z_k, rho_k again
  int pad_state;
  unsigned int ticket[4];
  int phase_runs[8];         // iterations started per phase 2 u_z + u_r
  // histories (device)
  double* delta_hist;        // [maxit + 2]
  unsigned char* prec_hist;  // [maxit + 1]
  double dring[kRing];       // delta_t at t % kRing
};
static_assert(sizeof(DevState) % 16 == 0, "state is copied in 16-byte words");

// Reduction tails work on a shared-memory copy of the state: the block loads
// it with one round of 16-byte loads (issued together with the partials'
// loads), thread 0 runs the scalar step at shared-memory latency, and the
// block writes it back.  Only the last block of a kernel touches the state
// after the kernel's start, so the copy is not raced.
__device__ __forceinline__ void state_load(DevState* s, const DevState* st) {
  const int4* src = reinterpret_cast<const int4*>(st);
  int4* dst = reinterpret_cast<int4*>(s);
  for (int i = threadIdx.x; i < (int)(sizeof(DevState) / 16); i += blockDim.x) dst[i] = __ldcg(src + i);
}
__device__ __forceinline__ void state_store(DevState* st, const DevState* s) {
  __syncthreads();
  const int4* src = reinterpret_cast<const int4*>(s);
  int4* dst = reinterpret_cast<int4*>(st);
  for (int i = threadIdx.x; i < (int)(sizeof(DevState) / 16); i += blockDim.x) dst[i] = src[i];
}

// delta_t from the ring, or from a full history array (selector replay)
struct RingHist {
  const DevState* s;
  __device__ __forceinline__ double operator()(int t) const { return s->dring[t & (kRing - 1)]; }
};
struct ArrayHist {
  const double* d;
  __device__ __forceinline__ double operator()(int t) const { return d[t]; }
};

// Precision pair check at kernel entry.  The loop graph repeats one pair's
// launch sequence `chunk` times; after the selector changes the pair inside a
// chunk, the rest of that chunk's launches find another pair here and do
// nothing (every kernel of an iteration checks the same pair, which only the
// update kernel's last block changes).  All blocks read the same state, so
// all return together and no reduction ticket is taken.
__device__ __forceinline__ bool phase_mismatch(const DevState* st, int uz, int ur) {
  return st->uz != uz || st->ur != ur;
}

// Entry of an iteration kernel: the block copies the state to shared memory
// in one round of loads (instead of a chain of dependent reads: the done
// flag, then the precision pair, then the scalars and buffer choices), and
// every thread reads its fields there.  False: the solve is done or the
// precision pair is not (uz, ur).
__device__ __forceinline__ bool state_enter(DevState* S, const DevState* st, int uz, int ur) {
  state_load(S, st);
  __syncthreads();
  return !S->done && !phase_mismatch(S, uz, ur);
}

// Matrix in sliced-ELL form: rows are grouped 32 per slice (one warp); the
// entries of a slice are stored column-major (entry j of row lane at
// off[s] + 32 j + lane), so the warp's loads of values and indices are
// contiguous.  Each row keeps its CSR entries in ascending column order,
// padded with (value 0, column = row) up to the slice width.  Column indices
// are int32 absolute or int16 offsets col - row (when every offset fits).
struct Sell {
  int64_t n, nslices;
  int maxw;              // largest slice width
  const long long* off;  // [nslices]
  const int* width;      // [nslices]
  const int* cabs;       // int32 absolute columns, or null
  const short* coff;     // int16 offsets, or null
  const double* v64;
  const float* v32;
  int stream_hint;       // matrix larger than L2's share: staged loads marked evict-first
  // slice-uniform offsets (int16 layout only, else null): pat[8 s + j] is the
  // column offset of entry j of every row of slice s, or pat[8 s] = kNoPat
  // when the rows of the slice differ (then coff holds them, as always)
  const short* pat;
  // uniform slices only: bit j of rmask[row] set iff entry j of the row is
  // one of its stored CSR entries (the others are the added zeros)
  const unsigned char* rmask;
};
constexpr short kNoPat = (short)-32768;
__device__ __forceinline__ bool slice_uniform(const Sell& A, int64_t s) {
  return A.pat != nullptr && A.pat[s * 8] != kNoPat;
}

// Scalar-side pieces of the algorithm, evaluated by one thread -------------

// Eq. (eta_k) with reading R3 (no estimate before k >= d; ||r_{-1}|| := ||r_0||).
template <class H>
__device__ __forceinline__ double eta_window_dev(H delta, int k, int d, double C) {
  if (k < d) return __longlong_as_double(0x7ff0000000000000ll);
  double eta = 0.0;
  double c3 = __dadd_rn(3.0, C), c2 = __dadd_rn(2.0, C);
  for (int t = k - d; t <= k; ++t) {
    double prev = (t >= 1) ? delta(t - 1) : delta(0);
    double term = __dmul_rn(AMPCG_EPS32, __dadd_rn(__dmul_rn(c3, prev), __dmul_rn(c2, delta(t))));
    eta = __dadd_rn(eta, term);
  }
  return eta;
}

// Eq. (linear criterion) with reading R3 and +inf when the rate is >= 1.
template <class H>
__device__ __forceinline__ double eta_linear_dev(H delta, int k, int ell, double C) {
  const double inf = __longlong_as_double(0x7ff0000000000000ll);
  if (k < ell || k < 1) return inf;
  double rho = pow(delta(k) / delta(k - ell), 1.0 / (double)ell);
  if (!(rho < 1.0)) return inf;
  double c = __dmul_rn(AMPCG_EPS32, __dadd_rn(5.0, __dmul_rn(2.0, C)));
  return __dmul_rn(c, delta(k - 1)) / __dadd_rn(1.0, -rho);
}

// ---------------------------------------------------------------------------
// The selector's comparisons without the slow scalar path.
//
// On B300 a dependent binary64 operation costs ~64 cycles, a division ~550
// and pow ~5800, and this scalar step sits on the critical path of every
// iteration (one thread of the last block).  Each comparison the selector
// makes is therefore first tried against precomputed brackets that settle it
// whenever the two sides differ by more than 1e-12 (u_z tests) or 1e-9
// (u_r test) relative -- margins far above the rounding errors of both the
// bracket and the binary64 evaluation -- and only a comparison inside the
// margin evaluates Eq. (precision_selector) / Eq. (linear criterion) in
// binary64 exactly as written.  The outcome is always that of the binary64
// evaluation; the brackets only skip work.

constexpr double kNuMargin = 1e-12;
constexpr double kEtaMargin = 1e-9;

// Brackets from nb, tol_nb, tau_zs, tau_zh, C (once per solve).
__device__ __forceinline__ void prep_selector(DevState* s) {
  s->inv_tol_nb = 1.0 / s->tol_nb;
  double zs = __dmul_rn(s->tau_zs, s->nb), zh = __dmul_rn(s->tau_zh, s->nb);
  s->tzs_lo = __dmul_rn(zs, 1.0 - kNuMargin);
  s->tzs_hi = __dmul_rn(zs, 1.0 + kNuMargin);
  s->tzh_lo = __dmul_rn(zh, 1.0 - kNuMargin);
  s->tzh_hi = __dmul_rn(zh, 1.0 + kNuMargin);
  s->c_lin = __dmul_rn(AMPCG_EPS32, __dadd_rn(5.0, __dmul_rn(2.0, s->C)));
}

// fl(delta / nb) >= tau
__device__ __forceinline__ bool nu_at_least(double delta, double nb, double tau, double lo, double hi) {
  if (delta > hi) return true;
  if (delta < lo) return false;
  return __ddiv_rn(delta, nb) >= tau;
}

// y^e for e >= 1 by repeated squaring
__device__ __forceinline__ double ipow(double y, int e) {
  double r = 1.0;
  while (e) {
    if (e & 1) r = __dmul_rn(r, y);
    y = __dmul_rn(y, y);
    e >>= 1;
  }
  return r;
}

// eta_k <= tol ||b|| for Eq. (linear criterion).  In exact arithmetic, with
// t = c delta_{k-1} / T and rho = (delta_k / delta_{k-ell})^(1/ell):
// eta_k <= T  <=>  rho <= 1 - t  <=>  delta_k <= (1 - t)^ell delta_{k-ell};
// and eta_k >= c delta_{k-1} > T whenever t > 1.
template <class H>
__device__ __forceinline__ bool linear_switch(const DevState* s, H delta, int k) {
  const int ell = s->ell;
  if (k < ell || k < 1) return false;   // eta_k = +inf (reading R3)
  double t = __dmul_rn(__dmul_rn(s->c_lin, delta(k - 1)), s->inv_tol_nb);
  if (t > 1.0 + kEtaMargin) return false;
  if (t < 1.0 - 1e-3) {
    double rhs = __dmul_rn(ipow(__dadd_rn(1.0, -t), ell), delta(k - ell));
    double dk = delta(k);
    if (dk < __dmul_rn(rhs, 1.0 - kEtaMargin)) return true;
    if (dk > __dmul_rn(rhs, 1.0 + kEtaMargin)) return false;
  }
  return eta_linear_dev(delta, k, ell, s->C) <= s->tol_nb;
}

// eta_k <= tol ||b|| for Eq. (eta_k).  eta_k = eps32 (c3 S1 + c2 S2) with
// S1 = sum of delta_{t-1}, S2 = sum of delta_t over the window: all terms are
// positive, so sums taken in any order are within (d + 4) u of the exact
// value, as is the binary64 evaluation of the formula in its own order; the
// bracket uses four independent partial sums (the exact-order evaluation costs
// a chain of ~4 (d + 1) dependent binary64 operations).
template <class H>
__device__ __forceinline__ bool window_switch(const DevState* s, H delta, int k) {
  const int d = s->d;
  if (k < d) return false;   // eta_k = +inf (reading R3)
  double a[4] = {0.0, 0.0, 0.0, 0.0}, b[4] = {0.0, 0.0, 0.0, 0.0};
  int t = k - d;
  for (; t + 3 <= k; t += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int tt = t + u;
      a[u] = __dadd_rn(a[u], (tt >= 1) ? delta(tt - 1) : delta(0));
      b[u] = __dadd_rn(b[u], delta(tt));
    }
  }
  for (; t <= k; ++t) {
    a[0] = __dadd_rn(a[0], (t >= 1) ? delta(t - 1) : delta(0));
    b[0] = __dadd_rn(b[0], delta(t));
  }
  const double s1 = __dadd_rn(__dadd_rn(a[0], a[1]), __dadd_rn(a[2], a[3]));
  const double s2 = __dadd_rn(__dadd_rn(b[0], b[1]), __dadd_rn(b[2], b[3]));
  const double c3 = __dadd_rn(3.0, s->C), c2 = __dadd_rn(2.0, s->C);
  const double eta = __dmul_rn(AMPCG_EPS32, __dadd_rn(__dmul_rn(c3, s1), __dmul_rn(c2, s2)));
  const double T = s->tol_nb;
  if (eta < __dmul_rn(T, 1.0 - kEtaMargin)) return true;
  if (eta > __dmul_rn(T, 1.0 + kEtaMargin)) return false;
  return eta_window_dev(delta, k, d, s->C) <= T;
}

// 2^e as binary64 / binary32 (round-to-nearest-even of the exact power),
// built from the bit pattern.
__device__ __forceinline__ double pow2_f64(int e) {
  if (e > 1023) return __longlong_as_double(0x7ff0000000000000ll);
  if (e >= -1022) return __longlong_as_double((long long)(e + 1023) << 52);
  if (e >= -1074) return __longlong_as_double(1ll << (e + 1074));
  return 0.0;
}
__device__ __forceinline__ float pow2_f32(int e) {
  if (e > 127) return __uint_as_float(0x7f800000u);
  if (e >= -126) return __uint_as_float((unsigned)(e + 127) << 23);
  if (e >= -149) return __uint_as_float(1u << (e + 149));
  return 0.f;
}

// ceil(log2 m) for a positive finite binary64 m, from its bit pattern.
__device__ __forceinline__ int ceil_log2(double m) {
  unsigned long long b = (unsigned long long)__double_as_longlong(m);
  int eb = (int)(b >> 52);
  unsigned long long f = b & 0x000FFFFFFFFFFFFFull;
  if (eb == 0) {                                  // subnormal: m = f 2^-1074
    int p = 63 - __clzll((long long)f);
    return p - 1074 + ((f & (f - 1ull)) ? 1 : 0);
  }
  return eb - 1023 + (f ? 1 : 0);
}

// omega_k (reading R5): NONE 1, L2 1/delta_k (as printed in Alg. 3), the
// power-of-two modes 2^-ceil(log2 m) for the given max|r| (none for m = 0 or
// non-finite).
__device__ __forceinline__ int omega_exponent(double m) {
  const bool have = m > 0.0 && m < __longlong_as_double(0x7ff0000000000000ll);
  return have ? -ceil_log2(m) : 0;
}
__device__ __forceinline__ void set_omega(DevState* st, double m) {
  double om = 1.0;
  int pow2 = 1, e = 0;
  if (st->scale == SCALE_L2) {
    om = 1.0 / st->delta;
    pow2 = 0;
  } else if (st->scale == SCALE_LINF_POW2 || st->scale == SCALE_LINF_POW2_LAG) {
    e = omega_exponent(m);
    om = pow2_f64(e);
  }
  st->omega = om;
  st->omega_f = pow2 ? pow2_f32(e) : __double2float_rn(om);
  st->omega_pow2 = pow2;
  st->omega_e = e;
}

// Decide the precisions of iteration st->k (Alg. 3, precision selection), the storage
// conversions they imply, and omega_k (reading R5).  Thread 0 of one block;
// hist(t) gives delta_t.  Eq. (precision_selector): u_z from nu_k and u0, u_r
// from eta_k (reading R2).  With the latch on, a u_r already at FP32 cannot
// change and eta_k is not evaluated.
template <class H>
__device__ void decide(DevState* st, H hist) {
  int k = st->k;
  int uz, ur;
  if (st->criterion == CRIT_FIXED) {
    uz = st->fixed_uz;
    ur = st->fixed_ur;
  } else {
    const double dk = hist(k);
    const int u0 = st->u0;
    if (nu_at_least(dk, st->nb, st->tau_zs, st->tzs_lo, st->tzs_hi)) uz = u0;
    else if (nu_at_least(dk, st->nb, st->tau_zh, st->tzh_lo, st->tzh_hi)) uz = (u0 > P32) ? u0 : P32;
    else uz = (u0 > P16) ? u0 : P16;
    bool sw;
    if (st->latch && st->ur == P32) sw = true;
    else if (st->criterion == CRIT_WINDOW) sw = window_switch(st, hist, k);
    else sw = linear_switch(st, hist, k);
    ur = sw ? P32 : P64;
    if (st->latch) {
      if (uz < st->uz) uz = st->uz;
      if (ur < st->ur) ur = st->ur;
    }
  }
  if (uz != st->uz && uz == P32 && st->switch_iter[0] < 0) st->switch_iter[0] = k;
  if (uz != st->uz && uz == P16 && st->switch_iter[1] < 0) st->switch_iter[1] = k;
  if (ur != st->ur && ur == P32 && st->switch_iter[2] < 0) st->switch_iter[2] = k;
  st->r_cast = (ur != st->ur);
  st->p_cast = (!st->first && uz != st->uz_p);
  st->uz = uz;
  st->ur = ur;
  if (st->prec_hist) st->prec_hist[k] = (unsigned char)((uz << 4) | ur);
  // omega_k: the lagged mode takes max|r_{k-1}| (reading R20; init sets
  // maxr_prev = max|r_0| for k = 0)
  st->omega_exact = 0;
  set_omega(st, st->scale == SCALE_LINF_POW2_LAG ? st->maxr_prev : st->maxr);
  // c = ceil(log2 max|r_k|) (none for max|r_k| = 0 or non-finite)
  const double mr = st->maxr;
  const bool have_c = mr > 0.0 && mr < __longlong_as_double(0x7ff0000000000000ll);
  const int cl = have_c ? ceil_log2(mr) : 0;
  // sigma_k = 2^-ceil(log2 max|r_k|) (clamped to binary32's normal range):
  // scales r in binary32 inner products so that their terms stay in range
  int se = have_c ? -cl : 0;
  se = se < -126 ? -126 : (se > 126 ? 126 : se);
  st->sig_e = se;
  st->sig_f = pow2_f32(se);
  st->inv_sig = pow2_f64(-se);
  st->inv_sig2 = pow2_f64(-2 * se);
}

// ---------------------------------------------------------------------------
// Work partition of the row and element loops, and how they load vectors.
// GridPart: the whole grid works on one system per launch; every vector a
// loop reads was written by an earlier launch, so any load path is valid
// (plain cached loads for gathers, the read-only path for streams).
// TeamPart (batched.cuh): one block runs a whole solve in one launch, and
// vectors written by other threads between barriers are loaded coherently.
struct GridPart {
  __device__ static __forceinline__ int64_t first() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
  __device__ static __forceinline__ int64_t count() { return (int64_t)gridDim.x * blockDim.x; }
  // warps in block order (the slice loops: a warp per slice or per run of slices)
  __device__ static __forceinline__ int64_t warp() { return first() >> 5; }
  __device__ static __forceinline__ int64_t warps() { return count() >> 5; }
  template <class T>
  __device__ static __forceinline__ T ldm(const T* p) { return *p; }
  template <int V, class T>
  __device__ static __forceinline__ void vldm(const T* p, T (&o)[V]) { vldg<V>(p, o); }
  // elements this thread itself reads and rewrites in the launch
  template <int V, class T>
  __device__ static __forceinline__ void vldo(const T* p, T (&o)[V]) { vld<V>(p, o); }
};

// ---------------------------------------------------------------------------
// Sparse product of one row.  A in precision UR, p stored in precision UZ;
// operands widened exactly to UR (or rounded, when u_z is the higher one),
// one fma per stored entry in ascending column order, accumulated in UR.

template <int UZ, int UR> struct PToR;
template <int UZ> struct PToR<UZ, P64> {
  static __device__ __forceinline__ double cv(typename Store<UZ>::T v) { return to_f64(v); }
};
template <> struct PToR<P64, P32> {
  static __device__ __forceinline__ float cv(double v) { return __double2float_rn(v); }
};
template <> struct PToR<P32, P32> {
  static __device__ __forceinline__ float cv(float v) { return v; }
};
template <> struct PToR<P16, P32> {
  static __device__ __forceinline__ float cv(__half v) { return h2f(v); }
};

template <int UR> __device__ __forceinline__ typename Store<UR>::T fma_r(typename Store<UR>::T a,
                                                                         typename Store<UR>::T b,
                                                                         typename Store<UR>::T c);
template <> __device__ __forceinline__ double fma_r<P64>(double a, double b, double c) { return fma(a, b, c); }
template <> __device__ __forceinline__ float fma_r<P32>(float a, float b, float c) { return __fmaf_rn(a, b, c); }

template <int UR> __device__ __forceinline__ const typename Store<UR>::T* mat_vals(const Sell& A);
template <> __device__ __forceinline__ const double* mat_vals<P64>(const Sell& A) { return A.v64; }
template <> __device__ __forceinline__ const float* mat_vals<P32>(const Sell& A) { return A.v32; }

template <int IT> __device__ __forceinline__ int col_at(const Sell& A, long long e, int row);
template <> __device__ __forceinline__ int col_at<0>(const Sell& A, long long e, int row) { return __ldg(A.cabs + e); }
template <> __device__ __forceinline__ int col_at<1>(const Sell& A, long long e, int row) {
  return row + (int)__ldg(A.coff + e);
}

// acc = fma(val_j, x_j, acc) over the w stored entries of one row (entry j at
// base + 32 j), in ascending order.  Values and columns are loaded 8 entries
// (4 for binary64) at a time and the next chunk's loads are issued before the
// current chunk's gathers, so a wide row (elasticity: ~80 entries) keeps
// 8-16 loads in flight instead of one.
template <int IT, class TA, class Acc, class Gather, class Fma>
__device__ __forceinline__ Acc row_sum_chunked(const Sell& A, const TA* __restrict__ va, long long base, int w,
                                               int row, Acc acc, Gather gather, Fma fmaop) {
  constexpr int CH = (sizeof(TA) == 8 || sizeof(Acc) == 8) ? 4 : 8;
  TA a[CH];
  int c[CH];
#pragma unroll
  for (int u = 0; u < CH; ++u) {
    a[u] = TA(0);
    c[u] = row;
    if (u < w) {
      a[u] = __ldg(va + base + 32 * u);
      c[u] = col_at<IT>(A, base + 32 * u, row);
    }
  }
  for (int j0 = 0; j0 < w; j0 += CH) {
    TA an[CH];
    int cn[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int j = j0 + CH + u;
      an[u] = TA(0);
      cn[u] = row;
      if (j < w) {
        an[u] = __ldg(va + base + 32 * j);
        cn[u] = col_at<IT>(A, base + 32 * j, row);
      }
    }
    decltype(gather(0)) g[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u)
      if (j0 + u < w) g[u] = gather(c[u]);
#pragma unroll
    for (int u = 0; u < CH; ++u)
      if (j0 + u < w) acc = fmaop(a[u], g[u], acc);
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      a[u] = an[u];
      c[u] = cn[u];
    }
  }
  return acc;
}

// acc = sum_j a_ij p_j over row `row` of slice s (lane = row % 32).
template <int UZ, int UR, int IT>
__device__ __forceinline__ typename Store<UR>::T sell_row(const Sell& A, int s, int lane, int row,
                                                          const typename Store<UZ>::T* __restrict__ p) {
  using TR = typename Store<UR>::T;
  const TR* __restrict__ va = mat_vals<UR>(A);
  long long base = __ldg(A.off + s) + lane;
  int w = __ldg(A.width + s);
  TR acc = (TR)0;
  if (w <= 8) {
    TR a[8];
    int c[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (j < w) {
        a[j] = __ldg(va + base + 32 * j);
        c[j] = col_at<IT>(A, base + 32 * j, row);
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (j < w) acc = fma_r<UR>(a[j], PToR<UZ, UR>::cv(p[c[j]]), acc);
    }
  } else {
    acc = row_sum_chunked<IT>(A, va, base, w, row, acc,
                              [=](int j) { return PToR<UZ, UR>::cv(p[j]); },
                              [](TR av, TR xv, TR s) { return fma_r<UR>(av, xv, s); });
  }
  return acc;
}

// FP64 fma-chain row product (initial and true residual, Alg. 3).
template <int IT, class Part = GridPart>
__device__ __forceinline__ double sell_row64(const Sell& A, int s, int lane, int row,
                                             const double* __restrict__ x) {
  long long base = __ldg(A.off + s) + lane;
  int w = __ldg(A.width + s);
  return row_sum_chunked<IT>(A, A.v64, base, w, row, 0.0, [=](int j) { return Part::ldm(x + j); },
                             [](double av, double xv, double t) { return fma(av, xv, t); });
}

// ---------------------------------------------------------------------------
// Buffers of the iteration.
struct Bufs {
  double* x;       // FP64 iterate
  const double* b; // FP64 right-hand side
  double* r64;
  float* r32;
  void* z;         // u_z storage
  void* p[2];      // double-buffered search direction (u_z storage)
  void* q;         // u_r storage
  double* t;       // FP64 scratch (true residual)
  const double* dinv64;
  const float* dinv32;
  const __half* dinv16;
  double* part;            // per-block partial sums [G * 4]
  unsigned long long* pmax; // per-block partial maxima [G]
  GridSumBarrier* bar;      // barriers of the cooperative launches, one per precision pair [6]
};

// Alg. 3 on the state copy: rho_k, its checks (reading R12) and
// beta_{k-1} = rho_k / rho_{k-1}; completes the storage conversions.  Under
// the lagged scale a non-finite rho_k (y_k overflowed u_z) is not final:
// omega_k becomes 2^-ceil(log2 max|r_k|) and s->redo asks the caller to form
// y_k, z_k and rho_k again (reading R20; once per iteration).
__device__ __forceinline__ void rho_step(DevState* s, double r) {
  s->rho = r;
  s->redo = 0;
  if (!isfinite(r) && s->scale == SCALE_LINF_POW2_LAG && !s->omega_exact) {
    s->omega_exact = 1;
    set_omega(s, s->maxr);
    s->redo = 1;
    return;
  }
  if (!isfinite(r)) { s->status = ST_NONFINITE; s->done = 1; return; }
  if (!(r > 0.0)) { s->status = ST_BREAKDOWN; s->done = 1; return; }
  double beta = s->first ? 0.0 : r / s->rho_prev;
  s->beta = beta;
  s->beta_f = __double2float_rn(beta);
  s->r_cast = 0;
  if (s->p_cast) {
    s->pcur ^= 1;
    s->uz_p = s->uz;
    s->p_cast = 0;
  }
}

// ---------------------------------------------------------------------------
// Initial residual r_0 = b - A x_0 (FP64), ||b||, ||r_0||, max|r_0|; the last
// block stores delta_0 and decides iteration 0.  One thread per row.
template <int IT, class Part = GridPart>
__device__ __forceinline__ void init_rows(const Sell& A, const Bufs& B, double (&v)[2],
                                          unsigned long long& mx) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = Part::warp();
  const int64_t nwarps = Part::warps();
  for (int64_t s = warp; s < A.nslices; s += nwarps) {
    int row = (int)s * 32 + lane;
    if (row < A.n) {
      double t = sell_row64<IT, Part>(A, (int)s, lane, row, B.x);
      double bi = Part::ldm(B.b + row);
      double ri = bi - t;
      B.r64[row] = ri;
      v[0] = fma(bi, bi, v[0]);
      v[1] = fma(ri, ri, v[1]);
      unsigned long long kk = abs_key(ri);
      mx = kk > mx ? kk : mx;
    }
  }
}

// Alg. 3 initialisation on the state copy: ||b||, delta_0, the stopping test and the
// decision for iteration 0; returns delta_0.
__device__ __forceinline__ double init_step(DevState* s, double bb, double rr, unsigned long long m) {
  double nb = sqrt(bb);
  double d0 = sqrt(rr);
  s->nb = nb;
  s->tol_nb = s->tol * nb;
  prep_selector(s);
  s->delta = d0;
  s->maxr = __longlong_as_double((long long)m);
  s->maxr_prev = s->maxr;
  s->z_ready = 0;
  s->dring[0] = d0;
  s->k = 0;
  s->done = 0;
  s->status = ST_NOT_CONVERGED;
  if (!isfinite(nb) || !isfinite(d0)) {
    s->status = ST_NONFINITE;
    s->done = 1;
  } else if (d0 <= s->tol_nb) {
    s->status = ST_OK;
    s->done = 1;
  } else if (s->maxit <= 0) {
    s->done = 1;
  } else {
    decide(s, RingHist{s});
  }
  return d0;
}

template <int IT>
__global__ void __launch_bounds__(256) k_init(Sell A, Bufs B, DevState* st) {
  double v[2] = {0.0, 0.0};
  unsigned long long mx = 0ull;
  init_rows<IT>(A, B, v, mx);
  block_sum<2>(v);
  mx = block_max(mx);
  if (threadIdx.x == 0) {
    B.part[blockIdx.x * 4 + 0] = v[0];
    B.part[blockIdx.x * 4 + 1] = v[1];
    B.pmax[blockIdx.x] = mx;
  }
  if (!last_block(&st->ticket[0])) return;
  __shared__ DevState S;
  state_load(&S, st);
  double vv[2];
  unsigned long long m = final_sum_max<2>(B.part, 4, B.pmax, gridDim.x, vv);
  double d0 = 0.0;
  if (threadIdx.x == 0) {
    S.ticket[0] = 0u;
    d0 = init_step(&S, vv[0], vv[1], m);
  }
  state_store(st, &S);
  if (threadIdx.x == 0) {
    S.delta_hist[0] = d0;
  }
}

// ---------------------------------------------------------------------------
// Elementwise kernels process V consecutive elements per thread and loop trip
// (V = 4 or 8 on the solver's buffers, which are padded to a multiple of 64
// elements so whole vectors stay in bounds; V = 1 on caller arrays).  Only the
// first m = min(V, n - i0) elements of a vector are used and stored.  The
// update and precondition kernels take V = 4 (measured 6-7% faster than 8:
// more loop trips per thread let warps drift apart, so loads of one overlap
// the FP64 work of another).

// Alg. 3 scaling and preconditioning of V consecutive elements starting at
// i0 (m of them in range), and their rho_k terms: r_k is read in u_r
// (converted once when u_r changed, reading R10), y_k = omega_k r_k is
// computed in u_r and stored in u_z (reading R6), z_k = M^-1 y_k in u_z
// (Jacobi: one rounding of dinv_i * y_i).  rho_k = r_k^T z_k: binary32
// compensated products when neither operand is binary64 (r scaled by the
// exact power of two sig_f; the block total is unscaled), else one FP64 fma
// per term.
struct PrecondScalars {
  int r_cast, pow2, oe;
  bool om_one;
  double om;
  float omf, sigf;
  __device__ __forceinline__ explicit PrecondScalars(const DevState* st)
      : r_cast(st->r_cast), pow2(st->omega_pow2), oe(st->omega_e),
        om_one(st->omega_pow2 && st->omega_e == 0), om(st->omega), omf(st->omega_f), sigf(st->sig_f) {}
  // The scalars of iteration k + 1 as the update step of iteration k knows
  // them: NONE (omega = 1); the lagged power of two 2^-ceil(log2 max|r_k|)
  // (reading R20); and for the exact power of two the same exponent as a
  // guess, kept only when max|r_{k+1}| turns out to have it (the caller
  // checks).  The binary32 dot-product scale stays sigma_k (a power of two
  // that only keeps the terms in range; the block totals are unscaled by it).
  __device__ __forceinline__ static PrecondScalars next(const DevState* st) {
    PrecondScalars c(st);
    const bool p2 = st->scale == SCALE_LINF_POW2_LAG || st->scale == SCALE_LINF_POW2;
    const int e = p2 ? omega_exponent(st->maxr) : 0;
    c.r_cast = 0;
    c.pow2 = 1;
    c.oe = e;
    c.om_one = e == 0;
    c.om = pow2_f64(e);
    c.omf = pow2_f32(e);
    return c;
  }
};

// D^-1 of V consecutive rows in u_z (Jacobi; nothing for M = none).
template <int UZ, int MT, int V>
__device__ __forceinline__ void dinv_load(const Bufs& B, int64_t i0, typename Store<UZ>::T (&dv)[V]) {
  if constexpr (MT != M_NONE) {
    if constexpr (UZ == P64) vldg<V>(B.dinv64 + i0, dv);
    else if constexpr (UZ == P32) vldg<V>(B.dinv32 + i0, dv);
    else vldg<V>(B.dinv16 + i0, dv);
  }
}

// y = omega r computed in u_r and stored in u_z (reading R6), z = M^-1 y in
// u_z (Jacobi: one rounding of dinv_i y_i, reading R16), for V elements held
// in registers (m of them in range), and their rho_k terms.
template <int UZ, int UR, int MT, int V>
__device__ __forceinline__ void precond_regs(const PrecondScalars& c, const typename Store<UR>::T (&r)[V],
                                             const typename Store<UZ>::T (&dv)[V], int m,
                                             typename Store<UZ>::T (&zz)[V], double& rho, Dot2& d2) {
  using TZ = typename Store<UZ>::T;
  constexpr bool kSmall = (UR != P64) && (UZ != P64);
#pragma unroll
  for (int j = 0; j < V; ++j) {
    TZ y;
    if constexpr (UR == P64) {
      if constexpr (UZ == P16) y = c.pow2 ? d2h_scaled(r[j], c.oe) : d2h(__dmul_rn(c.om, r[j]));
      else y = round_from_f64<UZ>(c.om_one ? r[j] : __dmul_rn(c.om, r[j]));
    } else {
      y = round_from_f32<UZ>(__fmul_rn(c.omf, r[j]));
    }
    if constexpr (MT == M_NONE) zz[j] = y;
    else if constexpr (UZ == P64) zz[j] = __dmul_rn(dv[j], y);
    else if constexpr (UZ == P32) zz[j] = __fmul_rn(dv[j], y);
    else zz[j] = __float2half_rn(__fmul_rn(h2f(dv[j]), h2f(y)));
    if (j < m) {
      if constexpr (kSmall) d2.add(__fmul_rn((float)r[j], c.sigf), (float)zz[j]);
      else rho = fma(to_f64(r[j]), to_f64(zz[j]), rho);
    }
  }
}

template <int UZ, int UR, int MT, int V, class Part>
__device__ __forceinline__ void precond_vec(const Bufs& B, const PrecondScalars& c, int64_t i0, int m,
                                            typename Store<UZ>::T (&zz)[V], double& rho, Dot2& d2) {
  using TZ = typename Store<UZ>::T;
  using TR = typename Store<UR>::T;
  alignas(16) TR r[V];
  if constexpr (UR == P64) {
    if (c.r_cast) {
      alignas(16) float t[V];
      Part::template vldo<V>(B.r32 + i0, t);
#pragma unroll
      for (int j = 0; j < V; ++j) r[j] = f2d(t[j]);
      vst<V>(B.r64 + i0, r, m);
    } else {
      Part::template vldo<V>(B.r64 + i0, r);
    }
  } else {
    if (c.r_cast) {
      alignas(16) double t[V];
      Part::template vldo<V>(B.r64 + i0, t);
#pragma unroll
      for (int j = 0; j < V; ++j) r[j] = __double2float_rn(t[j]);
      vst<V>(B.r32 + i0, r, m);
    } else {
      Part::template vldo<V>(B.r32 + i0, r);
    }
  }
  alignas(16) TZ dv[V];
  dinv_load<UZ, MT, V>(B, i0, dv);
  precond_regs<UZ, UR, MT, V>(c, r, dv, m, zz, rho, d2);
}

// Alg. 3 scaling, preconditioning and rho_k over the thread's vectors; z_k
// goes to its buffer.
template <int UZ, int UR, int MT, int V, class Part = GridPart>
__device__ __forceinline__ void precond_rows(const Bufs& B, int64_t n, const DevState* st,
                                             double& rho, Dot2& d2) {
  using TZ = typename Store<UZ>::T;
  TZ* __restrict__ z = (TZ*)B.z;
  const PrecondScalars c(st);
  const int64_t nv = (n + V - 1) / V;
  const int64_t stride = Part::count();
  for (int64_t v = Part::first(); v < nv; v += stride) {
    const int64_t i0 = v * V;
    const int m = (n - i0 < V) ? (int)(n - i0) : V;
    alignas(16) TZ zz[V];
    precond_vec<UZ, UR, MT, V, Part>(B, c, i0, m, zz, rho, d2);
    vst<V>(z + i0, zz, m);
  }
}

// p_{k-1} brought to the new u_z once, when u_z changed (the search direction p_k is computed
// in u_z); the converted copy goes to the other search-direction buffer.
template <int UZ, class Part = GridPart>
__device__ __forceinline__ void cast_p(const Bufs& B, int64_t n, const DevState* st) {
  using TZ = typename Store<UZ>::T;
  const int uz_p = st->uz_p;
  const int pc = st->pcur;
  const void* pold = pc ? B.p[1] : B.p[0];
  TZ* pnew = (TZ*)(pc ? B.p[0] : B.p[1]);
  const int64_t stride = Part::count();
  for (int64_t i = Part::first(); i < n; i += stride) {
    double pv;
    if (uz_p == P64) pv = ((const double*)pold)[i];
    else if (uz_p == P32) pv = f2d(((const float*)pold)[i]);
    else pv = h2d(((const __half*)pold)[i]);
    pnew[i] = round_from_f64<UZ>(pv);
  }
}

template <int UZ, int UR, int MT, int V, class Part = GridPart>
__device__ __forceinline__ void precond_and_cast(const Bufs& B, int64_t n, const DevState* st,
                                                 double& rho, Dot2& d2) {
  precond_rows<UZ, UR, MT, V, Part>(B, n, st, rho, d2);
  if (st->p_cast) cast_p<UZ, Part>(B, n, st);
}


// ---------------------------------------------------------------------------
// Alg. 3 search direction: p_k = z_k + beta_{k-1} p_{k-1} in u_z (p_0 = z_0).
// One element of p_k = z_k + beta p_{k-1} for binary32/binary16 storage:
// binary32 fma, rounded once into u_z (reading R7).
template <int UZ>
__device__ __forceinline__ typename Store<UZ>::T axpy_one(float bf, typename Store<UZ>::T pp,
                                                         typename Store<UZ>::T zz) {
  if constexpr (UZ == P32) return __fmaf_rn(bf, pp, zz);
  else return __float2half_rn(__fmaf_rn(bf, h2f(pp), h2f(zz)));
}

template <int UZ, int V, class Part = GridPart>
__device__ __forceinline__ void axpy_rows(const Bufs& B, int64_t n, const DevState* st) {
  using TZ = typename Store<UZ>::T;
  const TZ* __restrict__ z = (const TZ*)B.z;
  const int pc = st->pcur;
  const TZ* __restrict__ po = (const TZ*)(pc ? B.p[1] : B.p[0]);
  TZ* __restrict__ pn = (TZ*)(pc ? B.p[0] : B.p[1]);
  const int first = st->first;
  const double beta = st->beta;
  const float bf = st->beta_f;
  const int64_t nv = (n + V - 1) / V;
  const int64_t stride = Part::count();
  for (int64_t v = Part::first(); v < nv; v += stride) {
    const int64_t i0 = v * V;
    const int m = (n - i0 < V) ? (int)(n - i0) : V;
    alignas(16) TZ zz[V];
    alignas(16) TZ pp[V];
    Part::template vldm<V>(z + i0, zz);
    if (first) {
      vst<V>(pn + i0, zz, m);
      continue;
    }
    Part::template vldm<V>(po + i0, pp);
#pragma unroll
    for (int j = 0; j < V; ++j) {
      if constexpr (UZ == P64) pp[j] = fma(beta, pp[j], zz[j]);
      else pp[j] = axpy_one<UZ>(bf, pp[j], zz[j]);
    }
    vst<V>(pn + i0, pp, m);
  }
}

template <int UZ, int UR>
__global__ void __launch_bounds__(256) k_axpy(Bufs B, int64_t n, DevState* st) {
  __shared__ DevState S;
  if (!state_enter(&S, st, UZ, UR)) return;
  axpy_rows<UZ, 8>(B, n, &S);
}

// Scaling, preconditioning, rho_k, beta_{k-1} and the search direction in one
// cooperative launch (Jacobi or no preconditioner).  The blocks meet once, at
// a grid barrier between rho_k's partial sums and the direction update; then
// every block sums the partials in the same fixed order and runs the same
// scalar step on its copy of the state, so all hold the same beta_{k-1}, and
// block 0 writes the state back.  z_k of the first kZreg vectors of a thread
// stays in registers between the two halves (it is read nowhere else); the
// buffer carries any further ones.
constexpr int kZreg = 2;
template <int UZ, int UR, int MT>
__global__ void __launch_bounds__(256) k_precond_dir(Bufs B, int64_t n, DevState* st) {
  using TZ = typename Store<UZ>::T;
  constexpr int V = 4;
  constexpr bool kSmall = (UR != P64) && (UZ != P64);
  __shared__ DevState S;
  if (!state_enter(&S, st, UZ, UR)) return;
  TZ* __restrict__ z = (TZ*)B.z;
  const int64_t nv = (n + V - 1) / V;
  const int64_t stride = GridPart::count();
  const int64_t v0 = GridPart::first();
  alignas(16) TZ zr[kZreg][V];
  int nb = 0;
  // a second pass only when the lagged scale made rho_k non-finite (reading R20)
  for (int attempt = 0; attempt < 2; ++attempt) {
    const PrecondScalars c(&S);
    double rho = 0.0;
    Dot2 d2;
#pragma unroll
    for (int t = 0; t < kZreg; ++t) {
      const int64_t v = v0 + t * stride;
      if (v < nv) {
        const int64_t i0 = v * V;
        const int m = (n - i0 < V) ? (int)(n - i0) : V;
        precond_vec<UZ, UR, MT, V, GridPart>(B, c, i0, m, zr[t], rho, d2);
      }
    }
    for (int64_t v = v0 + kZreg * stride; v < nv; v += stride) {
      const int64_t i0 = v * V;
      const int m = (n - i0 < V) ? (int)(n - i0) : V;
      alignas(16) TZ zz[V];
      precond_vec<UZ, UR, MT, V, GridPart>(B, c, i0, m, zz, rho, d2);
      vst<V>(z + i0, zz, m);
    }
    if (S.p_cast) cast_p<UZ>(B, n, &S);
    double v[1];
    if constexpr (kSmall) {
      v[0] = block_sum_dot2(d2, S.inv_sig);
    } else {
      v[0] = rho;
      block_sum<1>(v);
    }
    double tot;
    unsigned long long unused;
    const bool ok = grid_reduce_barrier<1>(B.bar + 2 * UZ + UR, B.part, nullptr, nb, v[0], 0ull, tot, unused);
    if (threadIdx.x == 0) {
      if (ok) {
        rho_step(&S, tot);
      } else {
        S.status = ST_TIMEOUT;
        S.done = 1;
        S.redo = 0;
      }
    }
    __syncthreads();
    if (!S.redo) break;
  }
  if (threadIdx.x == 0) S.phase_runs[2 * UZ + UR] += 1;
  __syncthreads();
  if (!S.done) {
    // p_k = z_k + beta_{k-1} p_{k-1}; p_{k-1} may have been converted by
    // other blocks of this launch (cast_p), so it is read through L2
    const int pc = S.pcur;
    const TZ* __restrict__ po = (const TZ*)(pc ? B.p[1] : B.p[0]);
    TZ* __restrict__ pn = (TZ*)(pc ? B.p[0] : B.p[1]);
    const int first = S.first;
    const double beta = S.beta;
    const float bf = S.beta_f;
    auto dir = [&](int64_t i0, int m, const TZ (&zz)[V]) {
      if (first) {
        vst<V>(pn + i0, zz, m);
        return;
      }
      alignas(16) TZ pp[V];
      vldcg<V>(po + i0, pp);
#pragma unroll
      for (int j = 0; j < V; ++j) {
        if constexpr (UZ == P64) pp[j] = fma(beta, pp[j], zz[j]);
        else pp[j] = axpy_one<UZ>(bf, pp[j], zz[j]);
      }
      vst<V>(pn + i0, pp, m);
    };
#pragma unroll
    for (int t = 0; t < kZreg; ++t) {
      const int64_t v = v0 + t * stride;
      if (v < nv) {
        const int64_t i0 = v * V;
        dir(i0, (n - i0 < V) ? (int)(n - i0) : V, zr[t]);
      }
    }
    for (int64_t v = v0 + kZreg * stride; v < nv; v += stride) {
      const int64_t i0 = v * V;
      alignas(16) TZ zz[V];
      vld<V>(z + i0, zz);
      dir(i0, (n - i0 < V) ? (int)(n - i0) : V, zz);
    }
  }
  if (blockIdx.x == 0) state_store(st, &S);
}

// ---------------------------------------------------------------------------
// Alg. 3 matrix product: q_k = A p_k in u_r, gamma_k = q_k^T p_k (FP64),
// alpha_k = rho_k / gamma_k.  One thread per row of a warp's slice.
// ---------------------------------------------------------------------------
// Staged SpMV.  The matrix stream (values and column indices) is the bulk of
// the bytes; a warp owns a contiguous run of slices (floor or ceil of slices
// per warp), taken in chunks of at most 32 (one header per lane), whose data
// is one contiguous region, and copies it into
// shared memory with a K-stage cp.async pipeline (16-byte copies through L2
// only), so K-1 slices are in flight while the current slice's gathers and
// fmas run.  cp.async.wait_group is a hardware wait, not a spin loop.  Every
// copy is 16-byte aligned: slice offsets are multiples of 32 entries and a
// slice holds 32 * width entries.
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
// The same copy with an L2 eviction-priority hint (createpolicy).  A matrix
// streamed once per iteration and larger than L2 is marked evict-first, so
// that the iteration vectors (re-read every iteration) stay in L2.
__device__ __forceinline__ unsigned long long l2_policy_evict_first() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void cp_async16_hint(void* sdst, const void* gsrc, unsigned long long pol) {
  unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gsrc), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

constexpr int kStageW = 8;  // widest slice the staged path takes
// Stages in flight per warp: 4 for binary32 values; 2 for binary64, which
// keeps four blocks per SM (measured: the FP64-accumulating SpMV is 7% faster
// than with three stages and three blocks).
template <int UR> struct StageCfg { static constexpr int K = (UR == P64) ? 2 : 4; };
template <int IT> struct IdxT;
template <> struct IdxT<0> { using T = int; };
template <> struct IdxT<1> { using T = short; };

// Shared-memory bytes of the staged SpMV for a block of `warps` warps with K
// stages per warp.
template <int UR, int IT, int K = StageCfg<UR>::K>
constexpr int staged_smem_bytes(int warps = 8) {
  return warps * K * 32 * kStageW * (int)(sizeof(typename Store<UR>::T) + sizeof(typename IdxT<IT>::T));
}

template <int UZ, int UR, int IT, class Part = GridPart, int K = StageCfg<UR>::K>
__device__ __forceinline__ void spmv_rows_staged(const Sell& A, const Bufs& B, const DevState* st,
                                                 double& gam, Dot2& d2, unsigned char* smem) {
  using TZ = typename Store<UZ>::T;
  using TR = typename Store<UR>::T;
  using TI = typename IdxT<IT>::T;
  constexpr int SE = 32 * kStageW;  // entries per stage
  constexpr bool kSmall = (UR != P64) && (UZ != P64);
  const TZ* __restrict__ p = (const TZ*)(st->pcur ? B.p[0] : B.p[1]);
  TR* __restrict__ q = (TR*)B.q;
  const TR* __restrict__ va = mat_vals<UR>(A);
  const TI* __restrict__ ia = IT ? (const TI*)A.coff : (const TI*)A.cabs;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  TR* sv = (TR*)(smem + (size_t)wib * K * SE * (sizeof(TR) + sizeof(TI)));
  TI* si = (TI*)(sv + K * SE);
  const int64_t gw = Part::warp();
  const int64_t nw = Part::warps();
  // warp gw owns slices [gw S / W, (gw + 1) S / W): runs differ by at most
  // one slice, the longer ones spread evenly over the blocks (SMs)
  const int64_t s1 = (gw + 1) * A.nslices / nw;
  const bool hint = A.stream_hint != 0;
  const unsigned long long pol = hint ? l2_policy_evict_first() : 0ull;
  // slice-uniform offsets (int16 layout): such a slice stages its values only
  const bool upat = IT == 1 && A.pat != nullptr;
  // chunks of at most 32 slices (one header per lane); one chunk per warp
  // while the runs hold at most 32 slices (the persistent kernel on 148 SMs:
  // up to 4.8 M rows)
  for (int64_t s0 = gw * A.nslices / nw; s0 < s1; s0 += 32) {
    const int cnt = (int)(s1 - s0 < 32 ? s1 - s0 : 32);
    long long hoff = 0;
    int hw = 0;
    uint4 hp = make_uint4(0u, 0u, 0u, 0u);   // the slice's 8 offsets, 2 per word
    if (lane < cnt) {
      hoff = __ldg(A.off + s0 + lane);
      hw = __ldg(A.width + s0 + lane);
      if (upat) hp = __ldg(reinterpret_cast<const uint4*>(A.pat) + s0 + lane);
    }
    const bool hu = upat && (short)(hp.x & 0xffffu) != kNoPat;
    const unsigned umask = __ballot_sync(0xffffffffu, hu);   // bit t: slice s0 + t uniform
    auto issue = [&](int t) {
      if (t < cnt) {
        const long long o = __shfl_sync(0xffffffffu, hoff, t);
        const int w = __shfl_sync(0xffffffffu, hw, t);
        const int stg = t % K;
        const char* gv = (const char*)(va + o);
        char* dv = (char*)(sv + stg * SE);
        const int nv = 2 * w * (int)sizeof(TR);  // 16-byte chunks: 32 w sizeof(TR) / 16
  #pragma unroll
        for (int u = 0; u < kStageW * (int)sizeof(TR) / 16; ++u) {
          const int c = lane + 32 * u;
          if (c < nv) {
            if (hint) cp_async16_hint(dv + 16 * c, gv + 16 * c, pol);
            else cp_async16(dv + 16 * c, gv + 16 * c);
          }
        }
        const char* gi = (const char*)(ia + o);
        char* di = (char*)(si + stg * SE);
        const int ni = ((umask >> t) & 1u) ? 0 : 2 * w * (int)sizeof(TI);
  #pragma unroll
        for (int u = 0; u < (kStageW * (int)sizeof(TI) + 15) / 16; ++u) {
          const int c = lane + 32 * u;
          if (c < ni) {
            if (hint) cp_async16_hint(di + 16 * c, gi + 16 * c, pol);
            else cp_async16(di + 16 * c, gi + 16 * c);
          }
        }
      }
      cp_async_commit();
    };
#pragma unroll
    for (int t = 0; t < K - 1; ++t) issue(t);
    // one row's product over a slice held in stage stg (w entries, w known at
    // compile time: no per-entry predicates)
    auto rowprod = [&](auto wc, int stg, int64_t row, TR& acc, bool uni, const uint4& pw) {
      constexpr int W = decltype(wc)::value;
      const TR* sa = sv + stg * SE + lane;
      const TI* sc = si + stg * SE + lane;
      TR a[W];
      int cc[W];
      const unsigned pws[4] = {pw.x, pw.y, pw.z, pw.w};
#pragma unroll
      for (int j = 0; j < W; ++j) {
        a[j] = sa[32 * j];
        if (uni) cc[j] = (int)row + (int)(short)((pws[j >> 1] >> (16 * (j & 1))) & 0xffffu);
        else cc[j] = IT ? (int)row + (int)sc[32 * j] : (int)sc[32 * j];
      }
      TZ g[W];
#pragma unroll
      for (int j = 0; j < W; ++j) g[j] = Part::ldm(p + cc[j]);
      acc = (TR)0;
#pragma unroll
      for (int j = 0; j < W; ++j) acc = fma_r<UR>(a[j], PToR<UZ, UR>::cv(g[j]), acc);
    };
    auto finish = [&](int64_t row, TR acc) {
      q[row] = acc;
      const TZ pr = Part::ldm(p + row);
      if constexpr (kSmall) d2.add((float)acc, (float)pr);
      else gam = fma(to_f64(acc), to_f64(pr), gam);
    };
    // one slice, or two of equal width whose gathers then overlap
    auto dispatch = [&](int w, auto fn) {
      switch (w) {
        case 1: fn(std::integral_constant<int, 1>{}); break;
        case 2: fn(std::integral_constant<int, 2>{}); break;
        case 3: fn(std::integral_constant<int, 3>{}); break;
        case 4: fn(std::integral_constant<int, 4>{}); break;
        case 5: fn(std::integral_constant<int, 5>{}); break;
        case 6: fn(std::integral_constant<int, 6>{}); break;
        case 7: fn(std::integral_constant<int, 7>{}); break;
        default: fn(std::integral_constant<int, kStageW>{}); break;
      }
    };
    // Invariant at the top of a trip at slice t: groups 0 .. t + K - 2 issued
    // (each issue commits one group, group i holding slice i in stage i % K).
    auto pat_of = [&](int t) {
      uint4 v;
      v.x = __shfl_sync(0xffffffffu, hp.x, t);
      v.y = __shfl_sync(0xffffffffu, hp.y, t);
      v.z = __shfl_sync(0xffffffffu, hp.z, t);
      v.w = __shfl_sync(0xffffffffu, hp.w, t);
      return v;
    };
    for (int t = 0; t < cnt;) {
      const int w0 = __shfl_sync(0xffffffffu, hw, t);
      const int w1 = __shfl_sync(0xffffffffu, hw, t + 1 < cnt ? t + 1 : t);
      const int64_t row = (s0 + t) * 32 + lane;
      if (K >= 3 && t + 1 < cnt && w0 == w1 && (s0 + t + 2) * 32 <= A.n) {
        issue(t + K - 1);          // into the stage of slice t - 1 (consumed)
        cp_async_wait<K - 2>();    // slices t and t + 1 have landed
        __syncwarp();
        const bool u0 = (umask >> t) & 1u, u1 = (umask >> (t + 1)) & 1u;
        const uint4 p0 = upat ? pat_of(t) : hp, p1 = upat ? pat_of(t + 1) : hp;
        dispatch(w0, [&](auto wc) {
          TR acc0, acc1;
          rowprod(wc, t % K, row, acc0, u0, p0);
          rowprod(wc, (t + 1) % K, row + 32, acc1, u1, p1);
          finish(row, acc0);
          finish(row + 32, acc1);
        });
        __syncwarp();              // the stages are refilled by the next issues
        issue(t + K);              // into the stage of slice t (consumed)
        t += 2;
      } else {
        issue(t + K - 1);
        cp_async_wait<K - 1>();
        __syncwarp();
        const bool u0 = (umask >> t) & 1u;
        const uint4 p0 = upat ? pat_of(t) : hp;
        if (row < A.n) {
          dispatch(w0, [&](auto wc) {
            TR acc;
            rowprod(wc, t % K, row, acc, u0, p0);
            finish(row, acc);
          });
        }
        __syncwarp();              // the stage is refilled by the next trip's issue
        t += 1;
      }
    }
    cp_async_wait<0>();
    __syncwarp();    // the next chunk refills the stages
  }
}

// Each warp owns a contiguous run of slices; it loads the headers (offset,
// width) of up to 32 slices with one coalesced load and hands them out by
// shuffle, so a slice costs two dependent memory round trips (entries, then
// gathers) instead of three.
template <int UZ, int UR, int IT, class Part = GridPart>
__device__ __forceinline__ void spmv_rows(const Sell& A, const Bufs& B, const DevState* st,
                                          double& gam, Dot2& d2) {
  using TZ = typename Store<UZ>::T;
  using TR = typename Store<UR>::T;
  const TZ* __restrict__ p = (const TZ*)(st->pcur ? B.p[0] : B.p[1]);
  TR* __restrict__ q = (TR*)B.q;
  constexpr bool kSmall = (UR != P64) && (UZ != P64);
  const TR* __restrict__ va = mat_vals<UR>(A);
  const int lane = threadIdx.x & 31;
  const int64_t gw = Part::warp();
  const int64_t nw = Part::warps();
  const int64_t s0 = gw * A.nslices / nw;        // runs as in spmv_rows_staged
  const int64_t s1 = (gw + 1) * A.nslices / nw;
  for (int64_t sb = s0; sb < s1; sb += 32) {
    const int64_t sh = sb + lane;
    long long hoff = 0;
    int hw = 0;
    if (sh < s1) {
      hoff = __ldg(A.off + sh);
      hw = __ldg(A.width + sh);
    }
    const int cnt = (int)(s1 - sb < 32 ? s1 - sb : 32);
    for (int i = 0; i < cnt; ++i) {
      const long long base = __shfl_sync(0xffffffffu, hoff, i) + lane;
      const int w = __shfl_sync(0xffffffffu, hw, i);
      const int64_t row = (sb + i) * 32 + lane;
      if (row >= A.n) continue;
      TR acc = (TR)0;
      if (w <= 8) {
        TR a[8];
        int c[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (j < w) {
            a[j] = __ldg(va + base + 32 * j);
            c[j] = col_at<IT>(A, base + 32 * j, (int)row);
          }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (j < w) acc = fma_r<UR>(a[j], PToR<UZ, UR>::cv(Part::ldm(p + c[j])), acc);
      } else {
        acc = row_sum_chunked<IT>(A, va, base, w, (int)row, acc,
                                  [=](int j) { return PToR<UZ, UR>::cv(Part::ldm(p + j)); },
                                  [](TR av, TR xv, TR s) { return fma_r<UR>(av, xv, s); });
      }
      q[row] = acc;
      const TZ pr = Part::ldm(p + row);
      if constexpr (kSmall) d2.add((float)acc, (float)pr);
      else gam = fma(to_f64(acc), to_f64(pr), gam);
    }
  }
}

// Alg. 3 on the state copy: gamma_k, its checks (reading R12),
// alpha_k = rho_k / gamma_k.
__device__ __forceinline__ void gamma_step(DevState* s, double g) {
  s->gamma = g;
  if (!isfinite(g)) {
    s->status = ST_NONFINITE;
    s->done = 1;
  } else if (!(g > 0.0)) {
    s->status = ST_BREAKDOWN;
    s->done = 1;
  } else {
    double a = s->rho / g;
    s->alpha = a;
    s->alpha_f = __double2float_rn(a);
  }
}

// WIDE = false (every slice at most kStageW wide): the staged path, launched
// with staged_smem_bytes<UR, IT>() of dynamic shared memory.  WIDE = true:
// the direct path with chunked row sums, no dynamic shared memory (a kernel
// of its own, so the wide-row code does not take registers from the staged
// one).
template <int UZ, int UR, int IT, bool WIDE>
__global__ void __launch_bounds__(256, WIDE ? 3 : 4) k_spmv(Sell A, Bufs B, DevState* st) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ DevState S;
  if (!state_enter(&S, st, UZ, UR)) return;
  double gam = 0.0;
  Dot2 d2;
  if constexpr (WIDE) spmv_rows<UZ, UR, IT>(A, B, &S, gam, d2);
  else spmv_rows_staged<UZ, UR, IT>(A, B, &S, gam, d2, dsm);
  double v[1];
  if constexpr ((UR != P64) && (UZ != P64)) {
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

// ---------------------------------------------------------------------------
// Alg. 3 updates: x += alpha p (FP64), r -= alpha q (u_r),
// delta_{k+1} = ||r|| (FP64), max|r| (exact); last block: stopping test and
// the decision for iteration k+1.
template <int UZ, int UR, int V, class Part = GridPart>
__device__ __forceinline__ void update_rows(const Bufs& B, int64_t n, const DevState* st,
                                            double& rr, Dot2& d2, unsigned long long& mx) {
  using TZ = typename Store<UZ>::T;
  using TR = typename Store<UR>::T;
  const TZ* __restrict__ p = (const TZ*)(st->pcur ? B.p[0] : B.p[1]);
  const TR* __restrict__ q = (const TR*)B.q;
  TR* __restrict__ rv = UR == P64 ? (TR*)B.r64 : (TR*)B.r32;
  const double a = st->alpha;
  const float af = st->alpha_f;
  const float sigf = st->sig_f;
  const int64_t nv = (n + V - 1) / V;
  const int64_t stride = Part::count();
  for (int64_t v = Part::first(); v < nv; v += stride) {
    const int64_t i0 = v * V;
    const int m = (n - i0 < V) ? (int)(n - i0) : V;
    alignas(16) TZ pp[V];
    alignas(16) TR qq[V];
    alignas(16) TR rr_[V];
    alignas(16) double xx[V];
    Part::template vldm<V>(p + i0, pp);
    Part::template vldm<V>(q + i0, qq);
    Part::template vldo<V>(rv + i0, rr_);
    Part::template vldo<V>(B.x + i0, xx);
#pragma unroll
    for (int j = 0; j < V; ++j) {
      xx[j] = fma(a, to_f64(pp[j]), xx[j]);
      if constexpr (UR == P64) {
        rr_[j] = fma(-a, qq[j], rr_[j]);
        if (j < m) {
          rr = fma(rr_[j], rr_[j], rr);
          unsigned long long kk = abs_key(rr_[j]);
          mx = kk > mx ? kk : mx;
        }
      } else {
        rr_[j] = __fmaf_rn(-af, qq[j], rr_[j]);
        if (j < m) {
          float rs = __fmul_rn(rr_[j], sigf);
          d2.add(rs, rs);
          unsigned kk = __float_as_uint(rr_[j]) & 0x7fffffffu;   // order-preserving |r|
          mx = kk > mx ? kk : mx;
        }
      }
    }
    vst<V>(B.x + i0, xx, m);
    vst<V>(rv + i0, rr_, m);
  }
  // the max was taken over binary32 bit patterns; return it as a binary64 key
  if constexpr (UR != P64) mx = abs_key(__uint_as_float((unsigned)mx));
}

// update_rows, and in the same pass over the vectors the scaling and
// preconditioning of the new residual for iteration k + 1 with the scalars cn
// (PrecondScalars::next): z_{k+1} goes to its buffer and its rho_{k+1} terms
// to rho / d2z.  Valid when iteration k + 1 keeps the precision pair (the
// caller discards z_{k+1} otherwise).
template <int UZ, int UR, int MT, int V, class Part = GridPart>
__device__ __forceinline__ void update_precond_rows(const Bufs& B, int64_t n, const DevState* st,
                                                    const PrecondScalars& cn, double& rr, Dot2& d2,
                                                    unsigned long long& mx, double& rho, Dot2& d2z) {
  using TZ = typename Store<UZ>::T;
  using TR = typename Store<UR>::T;
  const TZ* __restrict__ p = (const TZ*)(st->pcur ? B.p[0] : B.p[1]);
  const TR* __restrict__ q = (const TR*)B.q;
  TR* __restrict__ rv = UR == P64 ? (TR*)B.r64 : (TR*)B.r32;
  TZ* __restrict__ z = (TZ*)B.z;
  const double a = st->alpha;
  const float af = st->alpha_f;
  const float sigf = st->sig_f;
  const int64_t nv = (n + V - 1) / V;
  const int64_t stride = Part::count();
  for (int64_t v = Part::first(); v < nv; v += stride) {
    const int64_t i0 = v * V;
    const int m = (n - i0 < V) ? (int)(n - i0) : V;
    alignas(16) TZ pp[V];
    alignas(16) TR qq[V];
    alignas(16) TR rr_[V];
    alignas(16) double xx[V];
    alignas(16) TZ dv[V];
    Part::template vldm<V>(p + i0, pp);
    Part::template vldm<V>(q + i0, qq);
    Part::template vldo<V>(rv + i0, rr_);
    Part::template vldo<V>(B.x + i0, xx);
    dinv_load<UZ, MT, V>(B, i0, dv);
#pragma unroll
    for (int j = 0; j < V; ++j) {
      xx[j] = fma(a, to_f64(pp[j]), xx[j]);
      if constexpr (UR == P64) {
        rr_[j] = fma(-a, qq[j], rr_[j]);
        if (j < m) {
          rr = fma(rr_[j], rr_[j], rr);
          unsigned long long kk = abs_key(rr_[j]);
          mx = kk > mx ? kk : mx;
        }
      } else {
        rr_[j] = __fmaf_rn(-af, qq[j], rr_[j]);
        if (j < m) {
          float rs = __fmul_rn(rr_[j], sigf);
          d2.add(rs, rs);
          unsigned kk = __float_as_uint(rr_[j]) & 0x7fffffffu;   // order-preserving |r|
          mx = kk > mx ? kk : mx;
        }
      }
    }
    vst<V>(B.x + i0, xx, m);
    vst<V>(rv + i0, rr_, m);
    alignas(16) TZ zz[V];
    precond_regs<UZ, UR, MT, V>(cn, rr_, dv, m, zz, rho, d2z);
    vst<V>(z + i0, zz, m);
  }
  if constexpr (UR != P64) mx = abs_key(__uint_as_float((unsigned)mx));
}

// Alg. 3 on the state copy: delta_{k+1}, the stopping test,
// k <- k + 1 and the decision for the new iteration; returns delta_{k+1}.
__device__ __forceinline__ double update_step(DevState* s, double rr, unsigned long long m) {
  double d = sqrt(rr);
  int k1 = s->k + 1;
  s->delta = d;
  s->maxr_prev = s->maxr;
  s->maxr = __longlong_as_double((long long)m);
  s->z_ready = 0;
  s->dring[k1 & (kRing - 1)] = d;
  s->rho_prev = s->rho;
  s->first = 0;
  s->pcur ^= 1;        // p_k is now the previous direction
  s->uz_p = s->uz;
  s->k = k1;
  if (!isfinite(d)) {
    s->status = ST_NONFINITE;
    s->done = 1;
  } else if (d <= s->tol_nb) {
    s->status = ST_OK;
    s->done = 1;
  } else if (k1 >= s->maxit) {
    s->status = ST_NOT_CONVERGED;
    s->done = 1;
  } else {
    decide(s, RingHist{s});
  }
  return d;
}

template <int UZ, int UR>
__global__ void __launch_bounds__(256) k_update(Bufs B, int64_t n, DevState* st) {
  __shared__ DevState S;
  if (!state_enter(&S, st, UZ, UR)) return;
  double rr = 0.0;
  Dot2 d2;
  unsigned long long mx = 0ull;
  update_rows<UZ, UR, 4>(B, n, &S, rr, d2, mx);
  double v[1];
  if constexpr (UR != P64) {
    v[0] = block_sum_dot2(d2, S.inv_sig2);
  } else {
    v[0] = rr;
    block_sum<1>(v);
  }
  mx = block_max(mx);
  if (threadIdx.x == 0) {
    B.part[blockIdx.x] = v[0];
    B.pmax[blockIdx.x] = mx;
  }
  if (!last_block(&st->ticket[2])) return;
  state_load(&S, st);
  double tot[1];
  unsigned long long m = final_sum_max<1>(B.part, 1, B.pmax, gridDim.x, tot);
  double d = 0.0;
  int k1 = 0;
  if (threadIdx.x == 0) {
    S.ticket[2] = 0u;
    d = update_step(&S, tot[0], m);
    k1 = S.k;
  }
  state_store(st, &S);
  if (threadIdx.x == 0) S.delta_hist[k1] = d;
}

// ---------------------------------------------------------------------------
// The iteration loop of one precision pair as one cooperative launch (Jacobi
// or no preconditioner, slices at most kStageW wide): up to `iters`
// iterations of Alg. 3 on the same row loops as the kernels above, every block
// holding its own copy of the state.  The four grid-wide dependences of an
// iteration -- rho_k, p_k before the SpMV's gathers, gamma_k, and delta_{k+1}
// with max|r| -- are grid barriers whose last arriving block sums the
// partials (grid_reduce_barrier); every block then runs the same scalar step
// on its copy, so all agree on beta, alpha, the stop and the next
// precisions.  The launch ends after `iters` iterations, at the stop, or when
// the selector picks another pair; block 0 writes the state back (only it
// writes the histories).  Data that other blocks write during the launch is
// read through L2 (LoopPart), never through the read-only path.
struct LoopPart {
  // Rank of the thread in the grid-stride loops over rows or vectors, warps
  // interleaved across the blocks (warp w of block b is warp w G + b, G
  // blocks): a loop whose trip count is not the same for every thread gives
  // its extra trips to the first warps of every block rather than to whole
  // blocks, so the work per SM (the FP64 pipe is an SM's own) differs by at
  // most a warp's.  Each warp still covers 32 consecutive indices.
  __device__ static __forceinline__ int64_t first() {
    return ((int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32 + (threadIdx.x & 31);
  }
  __device__ static __forceinline__ int64_t count() { return (int64_t)gridDim.x * blockDim.x; }
  // warps in block order (the staged SpMV: each warp a contiguous run of slices)
  __device__ static __forceinline__ int64_t warp() { return ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
  __device__ static __forceinline__ int64_t warps() { return count() >> 5; }
  // the loads carry an L2 evict-last hint: the vectors stay in L2 across
  // iterations while the matrix streams through (evict-first)
  template <class T>
  __device__ static __forceinline__ T ldm(const T* p) { return ld_keep(p, l2_policy_evict_last()); }
  template <int V, class T>
  __device__ static __forceinline__ void vldm(const T* p, T (&o)[V]) { vld_keep<V>(p, o, l2_policy_evict_last()); }
  template <int V, class T>
  __device__ static __forceinline__ void vldo(const T* p, T (&o)[V]) { vld_keep<V>(p, o, l2_policy_evict_last()); }
};

// One block of kLoopBlock threads per SM: fewer blocks meet at each grid
// barrier (its arrivals and polls contend on one word), the same registers
// and shared memory per SM as four blocks of 256.  The staged SpMV's stages
// per warp are capped so that the block's stages fit in 200 KB.
constexpr int kLoopBlock = 1024;
template <int UR, int IT> struct LoopStageCfg {
  static constexpr int kPer = (kLoopBlock / 32) * 32 * kStageW *
                              (int)(sizeof(typename Store<UR>::T) + sizeof(typename IdxT<IT>::T));
  static constexpr int K = StageCfg<UR>::K < (200 * 1024) / kPer ? StageCfg<UR>::K : (200 * 1024) / kPer;
  static constexpr int kBytes = K * kPer;
};
template <int UZ, int UR, int MT, int IT, bool FUSED>
__global__ void __launch_bounds__(kLoopBlock, 1) k_loop(Sell A, Bufs B, int64_t n, DevState* st, int iters) {
  using TZ = typename Store<UZ>::T;
  using Part = LoopPart;
  constexpr int V = 4;                         // update
  constexpr int VZ = (UZ == P64) ? 4 : 8;      // precondition and direction
  constexpr bool kSmall = (UR != P64) && (UZ != P64);
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ DevState S;
  if (!state_enter(&S, st, UZ, UR)) return;
  if (blockIdx.x != 0 && threadIdx.x == 0) S.prec_hist = nullptr;   // block 0 records the choices
  GridSumBarrier* bar = B.bar + 6 + 2 * UZ + UR;
  TZ* __restrict__ z = (TZ*)B.z;
  const int64_t nvz = (n + VZ - 1) / VZ;
  const int64_t stride = Part::count();
  const int64_t v0 = Part::first();
  // FUSED (scale modes whose omega_{k+1} is known before delta_{k+1} is
  // reduced: no scaling, or the lagged power of two of reading R20): the
  // update step of iteration k also forms z_{k+1} and rho_{k+1}, reduced
  // together with delta_{k+1}: three grid barriers per iteration (p_k,
  // gamma_k, delta_{k+1} + rho_{k+1}) instead of four.  The head step
  // (scaling, preconditioning, rho_k on their own) then runs only after a
  // precision change, a residual replacement, at the first iteration, or to
  // retry a non-finite rho_k with the exact power of two.  A template
  // parameter rather than a run-time branch: one kernel holding both update
  // steps spilled 112-172 bytes of registers against 32-100.
  constexpr bool fused = FUSED;
  // z_k of the first kZr vectors of a thread kept in registers from the head
  // step to the direction step (the four-barrier form, whose every iteration
  // runs the head step); the three-barrier form runs it only now and then and
  // passes z_k through its buffer, which leaves the registers to the rest
  constexpr int kZr = FUSED ? 0 : kZreg;
  constexpr int kZa = kZr > 0 ? kZr : 1;
  double tot[2] = {0.0, 0.0};
  unsigned long long mtot = 0ull;
  bool ok = true;
  int nb = 0;   // barriers passed in this launch
  for (int it = 0; it < iters; ++it) {
    alignas(16) TZ zr[kZa][VZ];
    alignas(16) TZ pr[kZa][VZ];
    bool have = false;   // z_k of the first kZr vectors of the thread in registers
    bool pre = false;    // and p_{k-1} of those vectors
    if (!S.z_ready) {
      // Alg. 3: scaling, preconditioning, rho_k and beta_{k-1}; with binary16
      // storage p_{k-1} of the register-held vectors is loaded before the
      // barrier (it does not depend on beta_{k-1}; not when it is converted)
      {
        pre = kZr > 0 && (UZ == P16) && !S.p_cast && !S.first;
        const PrecondScalars c(&S);
        double rho = 0.0;
        Dot2 d2;
#pragma unroll
        for (int t = 0; t < kZr; ++t) {
          const int64_t v = v0 + t * stride;
          if (v < nvz) {
            const int64_t i0 = v * VZ;
            precond_vec<UZ, UR, MT, VZ, Part>(B, c, i0, (n - i0 < VZ) ? (int)(n - i0) : VZ, zr[t], rho, d2);
          }
        }
        if constexpr (UZ == P16) {
          if (pre) {
            const TZ* po = (const TZ*)(S.pcur ? B.p[1] : B.p[0]);
#pragma unroll
            for (int t = 0; t < kZr; ++t) {
              const int64_t v = v0 + t * stride;
              if (v < nvz) vldcg<VZ>(po + v * VZ, pr[t]);
            }
          }
        }
        for (int64_t v = v0 + kZr * stride; v < nvz; v += stride) {
          const int64_t i0 = v * VZ;
          const int m = (n - i0 < VZ) ? (int)(n - i0) : VZ;
          alignas(16) TZ zz[VZ];
          precond_vec<UZ, UR, MT, VZ, Part>(B, c, i0, m, zz, rho, d2);
          vst<VZ>(z + i0, zz, m);
        }
        if (S.p_cast) cast_p<UZ, Part>(B, n, &S);
        double v[1];
        if constexpr (kSmall) {
          v[0] = block_sum_dot2(d2, S.inv_sig);
        } else {
          v[0] = rho;
          block_sum_wide<1>(v);
        }
        ok = grid_reduce_barrier<1>(bar, B.part, nullptr, nb, v[0], 0ull, tot[0], mtot);
        if (!ok) break;
        if (threadIdx.x == 0) rho_step(&S, tot[0]);
        __syncthreads();
      }
      if (!ok || S.done) break;
      if (S.redo) {   // omega_k is now the exact power of two (reading R20): the head again
        --it;
        continue;
      }
      have = kZr > 0;
    }
    if (threadIdx.x == 0) S.phase_runs[2 * UZ + UR] += 1;
    // Alg. 3: search direction p_k = z_k + beta_{k-1} p_{k-1}
    {
      const int pc = S.pcur;
      const TZ* __restrict__ po = (const TZ*)(pc ? B.p[1] : B.p[0]);
      TZ* __restrict__ pn = (TZ*)(pc ? B.p[0] : B.p[1]);
      const int first = S.first;
      const double beta = S.beta;
      const float bf = S.beta_f;
      auto dir = [&](int64_t i0, int m, const TZ (&zz)[VZ], const TZ (&pp0)[VZ], bool have_p) {
        if (first) {
          vst<VZ>(pn + i0, zz, m);
          return;
        }
        alignas(16) TZ pp[VZ];
        if (have_p) {
#pragma unroll
          for (int j = 0; j < VZ; ++j) pp[j] = pp0[j];
        } else {
          vldcg<VZ>(po + i0, pp);
        }
#pragma unroll
        for (int j = 0; j < VZ; ++j) {
          if constexpr (UZ == P64) pp[j] = fma(beta, pp[j], zz[j]);
          else pp[j] = axpy_one<UZ>(bf, pp[j], zz[j]);
        }
        vst<VZ>(pn + i0, pp, m);
      };
      if (have) {
#pragma unroll
        for (int t = 0; t < kZr; ++t) {
          const int64_t v = v0 + t * stride;
          if (v < nvz) {
            const int64_t i0 = v * VZ;
            dir(i0, (n - i0 < VZ) ? (int)(n - i0) : VZ, zr[t], pr[t], pre);
          }
        }
      }
      // z_k of the other vectors (all of them when the previous update step
      // formed z_k) is in its buffer, written by other threads before a barrier
      for (int64_t v = v0 + (have ? kZr * stride : 0); v < nvz; v += stride) {
        const int64_t i0 = v * VZ;
        alignas(16) TZ zz[VZ];
        vldcg<VZ>(z + i0, zz);
        dir(i0, (n - i0 < VZ) ? (int)(n - i0) : VZ, zz, zz, false);
      }
      ok = grid_reduce_barrier<0>(bar, nullptr, nullptr, nb, 0.0, 0ull, tot[0], mtot);   // p_k before the gathers
      if (!ok) break;
    }
    // Alg. 3: q_k = A p_k, gamma_k, alpha_k
    {
      double gam = 0.0;
      Dot2 d2;
      spmv_rows_staged<UZ, UR, IT, Part, LoopStageCfg<UR, IT>::K>(A, B, &S, gam, d2, dsm);
      double v[1];
      if constexpr (kSmall) {
        v[0] = block_sum_dot2(d2, 1.0);
      } else {
        v[0] = gam;
        block_sum_wide<1>(v);
      }
      ok = grid_reduce_barrier<1>(bar, B.part, nullptr, nb, v[0], 0ull, tot[0], mtot);
      if (!ok) break;
      if (threadIdx.x == 0) gamma_step(&S, tot[0]);
      __syncthreads();
      if (S.done) break;
    }
    // Alg. 3: x and r updates, delta_{k+1}, stopping test, next precisions;
    // fused: also z_{k+1} and rho_{k+1}
    {
      double rr = 0.0, rho = 0.0;
      Dot2 d2, d2z;
      unsigned long long mx = 0ull;
      if constexpr (fused) {
        const PrecondScalars cn = PrecondScalars::next(&S);
        update_precond_rows<UZ, UR, MT, V, Part>(B, n, &S, cn, rr, d2, mx, rho, d2z);
      } else {
        update_rows<UZ, UR, V, Part>(B, n, &S, rr, d2, mx);
      }
      // block totals of ||r||^2 (and rho_{k+1}) with max|r|, one pass where
      // the operand types allow
      double v[2] = {0.0, 0.0};
      if constexpr (kSmall) {
        if constexpr (fused) {
          Dot2 dd[2] = {d2, d2z};
          const double sc[2] = {S.inv_sig2, S.inv_sig};
          block_sums_dot2_max<2>(dd, sc, v, mx);
        } else {
          Dot2 dd[1] = {d2};
          const double sc[1] = {S.inv_sig2};
          double w[1];
          block_sums_dot2_max<1>(dd, sc, w, mx);
          v[0] = w[0];
        }
      } else if constexpr (UR == P64) {
        v[0] = rr;
        v[1] = rho;
        if constexpr (fused) {
          block_sum_wide_max<2>(v, mx);
        } else {
          double w[1] = {v[0]};
          block_sum_wide_max<1>(w, mx);
          v[0] = w[0];
        }
      } else {
        // u_z = FP64, u_r = FP32: ||r||^2 by Dot2, rho_{k+1} in binary64
        v[0] = block_sum_dot2(d2, S.inv_sig2);
        if constexpr (fused) {
          double w[1] = {rho};
          block_sum_wide<1>(w);
          v[1] = w[0];
        }
        mx = block_max(mx);
      }
      if constexpr (fused) ok = grid_barrier_sums<2, true>(bar, B.part, B.pmax, nb, v, mx, tot, mtot, kBarrierSpin);
      else ok = grid_barrier_sums<1, true>(bar, B.part, B.pmax, nb, v, mx, tot, mtot, kBarrierSpin);
      if (!ok) break;
      if (threadIdx.x == 0) {
        const double d = update_step(&S, tot[0], mtot);
        if (blockIdx.x == 0) S.delta_hist[S.k] = d;
        // the pair is kept: z_{k+1} and rho_{k+1} stand (or are retried by
        // the head step with the exact power of two).  Under the exact power
        // of two they were formed with the exponent of max|r_k|: they are the
        // exact scale's own (the same omega and sigma, so the same bits of
        // z) when max|r_{k+1}| has that exponent, else the head step forms
        // them again
        if (FUSED && !S.done && S.uz == UZ && S.ur == UR &&
            (S.scale != SCALE_LINF_POW2 || S.omega_e == omega_exponent(S.maxr_prev))) {
          rho_step(&S, tot[1]);
          S.z_ready = S.redo ? 0 : 1;
        }
      }
      __syncthreads();
      if (S.done || S.uz != UZ || S.ur != UR) break;
    }
  }
  if (!ok && threadIdx.x == 0) {
    S.status = ST_TIMEOUT;
    S.done = 1;
  }
  if (blockIdx.x == 0) state_store(st, &S);
}

// The staged SpMV of k_loop on its own, launched with k_loop's grid and
// shared memory, so its work split (each warp a contiguous run of
// floor or ceil(nslices / warps) slices, LoopStageCfg stages per warp, the two-slice
// overlapped trip, the L2 hint of the matrix stream) is the one the solve
// runs: q = A p in u_r; part[b] = block b's partial of gamma = q^T p.  B.p[0]
// and B.p[1] both hold p.  For parity tests of that code path.
template <int UZ, int UR, int IT>
__global__ void __launch_bounds__(kLoopBlock, 1) k_spmv_loop_step(Sell A, Bufs B, const DevState* st) {
  extern __shared__ __align__(16) unsigned char dsm[];
  constexpr bool kSmall = (UR != P64) && (UZ != P64);
  double gam = 0.0;
  Dot2 d2;
  spmv_rows_staged<UZ, UR, IT, LoopPart, LoopStageCfg<UR, IT>::K>(A, B, st, gam, d2, dsm);
  double v[1];
  if constexpr (kSmall) {
    v[0] = block_sum_dot2(d2, 1.0);
  } else {
    v[0] = gam;
    block_sum_wide<1>(v);
  }
  if (threadIdx.x == 0) B.part[blockIdx.x] = v[0];
}

// Loop graph control (one thread each).  The outer loop picks the precision
// pair's body with a SWITCH; the body repeats chunks of that pair's
// iterations in an inner loop while the pair stays current, so a SWITCH is
// evaluated once per precision change rather than once per iteration.

// Sets the SWITCH value of an outer-loop body: the current pair 2 u_z + u_r.
#ifndef AMPCG_INSTANTIATION_UNIT
__global__ void k_phase(DevState* st, cudaGraphConditionalHandle h) {
  cudaGraphSetConditional(h, st->done ? AMPCG_PHASE_NONE : 2 * st->uz + st->ur);
}
#endif

// End of an inner-loop chunk of pair ph: continue while the solve runs and
// the pair is still ph.  A chunk that ends without the iteration counter
// having advanced (which the dispatch never produces: the SWITCH chose ph
// from the same state) stops the solve with an internal error, so the inner
// loop ends within maxit chunks.
#ifndef AMPCG_INSTANTIATION_UNIT
__global__ void k_chunk_ctl(DevState* st, cudaGraphConditionalHandle h, int ph) {
  st->chunk_runs[ph] += 1;
  if (!st->done && st->k == st->k_chunk) {
    st->status = ST_INTERNAL;
    st->done = 1;
  }
  st->k_chunk = st->k;
  cudaGraphSetConditional(h, (!st->done && 2 * st->uz + st->ur == ph) ? 1u : 0u);
}
#endif

// Sets the condition of the outer loop; the same progress check per body.
#ifndef AMPCG_INSTANTIATION_UNIT
__global__ void k_loop_ctl(DevState* st, cudaGraphConditionalHandle h) {
  st->loop_runs += 1;
  if (!st->done && st->k == st->k_body) {
    st->status = ST_INTERNAL;
    st->done = 1;
  }
  st->k_body = st->k;
  cudaGraphSetConditional(h, st->done ? 0u : 1u);
}
#endif

// ---------------------------------------------------------------------------
// True residual t = b - A x in FP64 and ||t|| / ||b|| (exit verification).
template <int IT, class Part = GridPart>
__device__ __forceinline__ void true_res_rows(const Sell& A, const Bufs& B, double (&v)[1]) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = Part::warp();
  const int64_t nwarps = Part::warps();
  for (int64_t s = warp; s < A.nslices; s += nwarps) {
    int row = (int)s * 32 + lane;
    if (row < A.n) {
      double t = Part::ldm(B.b + row) - sell_row64<IT, Part>(A, (int)s, lane, row, B.x);
      B.t[row] = t;
      v[0] = fma(t, t, v[0]);
    }
  }
}

template <int IT>
__global__ void __launch_bounds__(256) k_true_residual(Sell A, Bufs B, DevState* st) {
  double v[1] = {0.0};
  true_res_rows<IT>(A, B, v);
  block_sum<1>(v);
  if (threadIdx.x == 0) B.part[blockIdx.x] = v[0];
  if (!last_block(&st->ticket[3])) return;
  __shared__ DevState S;
  state_load(&S, st);
  double tot[1];
  final_sum<1>(B.part, gridDim.x, 1, tot);
  if (threadIdx.x == 0) {
    S.ticket[3] = 0u;
    S.true_relres = sqrt(tot[0]) / S.nb;
  }
  state_store(st, &S);
}

// Residual replacement (reading R9): r <- round_ur(t), delta, max|r|; the
// solve continues from iteration st->k if the new residual misses tol.
template <class Part = GridPart>
__device__ __forceinline__ void refresh_rows(const Bufs& B, int64_t n, const DevState* st, double& rr,
                                             unsigned long long& mx) {
  const int ur = st->ur;
  const int64_t stride = Part::count();
  for (int64_t i = Part::first(); i < n; i += stride) {
    double t = Part::ldm(B.t + i);
    double rv;
    if (ur == P64) { rv = t; B.r64[i] = t; }
    else { float f = __double2float_rn(t); B.r32[i] = f; rv = f2d(f); }
    rr = fma(rv, rv, rr);
    unsigned long long kk = abs_key(rv);
    mx = kk > mx ? kk : mx;
  }
}

// Reading R9 on the state copy: the replaced residual's norm, the stopping
// test, and the decision for iteration k; returns the new delta_k.
__device__ __forceinline__ double refresh_step(DevState* s, double rr, unsigned long long m) {
  double d = sqrt(rr);
  int k = s->k;
  s->delta = d;
  s->maxr = __longlong_as_double((long long)m);
  s->z_ready = 0;
  s->dring[k & (kRing - 1)] = d;
  s->refreshes += 1;
  if (d <= s->tol_nb) {
    s->status = ST_OK;
    s->done = 1;
  } else {
    s->status = ST_NOT_CONVERGED;
    s->done = 0;
    decide(s, RingHist{s});
  }
  return d;
}

#ifndef AMPCG_INSTANTIATION_UNIT
__global__ void __launch_bounds__(256) k_refresh(Bufs B, int64_t n, DevState* st) {
  double rr = 0.0;
  unsigned long long mx = 0ull;
  refresh_rows(B, n, st, rr, mx);
  double v[1] = {rr};
  block_sum<1>(v);
  mx = block_max(mx);
  if (threadIdx.x == 0) {
    B.part[blockIdx.x] = v[0];
    B.pmax[blockIdx.x] = mx;
  }
  if (!last_block(&st->ticket[3])) return;
  __shared__ DevState S;
  state_load(&S, st);
  double tot[1];
  unsigned long long m = final_sum_max<1>(B.part, 1, B.pmax, gridDim.x, tot);
  double d = 0.0;
  int k = 0;
  if (threadIdx.x == 0) {
    S.ticket[3] = 0u;
    k = S.k;
    d = refresh_step(&S, tot[0], m);
  }
  state_store(st, &S);
  if (threadIdx.x == 0) {
    S.delta_hist[k] = d;
  }
}
#endif

// ---------------------------------------------------------------------------
// Create-time preparation (a1): CSR -> sliced layout, value copies, diagonal.

// Per row: structure checks, row length, diagonal, max |col - row|.
// flags bit 0: bad rowptr; bit 1: column out of range / not increasing;
// bit 2: diagonal missing or <= 0; bit 3: non-finite value.
#ifndef AMPCG_INSTANTIATION_UNIT
__global__ void k_csr_scan_rows(int64_t n, int64_t nnz, const int* rowptr, const int* col,
                                const double* val, int* rowlen, double* diag, int* flags,
                                int* maxoff) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = rowptr[i], b = rowptr[i + 1];
  int f = 0;
  if (a < 0 || b < a || b > nnz || (i == 0 && a != 0) || (i == n - 1 && b != nnz)) {
    atomicOr(flags, 1);
    rowlen[i] = 0;
    diag[i] = 0.0;
    return;
  }
  double dg = 0.0;
  int prev = -1, mo = 0;
  for (int k = a; k < b; ++k) {
    int c = col[k];
    double v = val[k];
    if (c < 0 || c >= n || c <= prev) f |= 2;
    if (!isfinite(v)) f |= 8;
    if (c == i) dg = v;
    int o = c - (int)i;
    o = o < 0 ? -o : o;
    mo = o > mo ? o : mo;
    prev = c;
  }
  if (!(dg > 0.0)) f |= 4;
  if (f) atomicOr(flags, f);
  rowlen[i] = b - a;
  diag[i] = dg;
  atomicMax(maxoff, mo);
}
#endif

#ifndef AMPCG_INSTANTIATION_UNIT
__global__ void k_slice_width(int64_t n, int64_t nslices, const int* rowlen, int* width) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nslices) return;
  int w = 0;
  for (int l = 0; l < 32; ++l) {
    int64_t r = s * 32 + l;
    if (r < n) w = rowlen[r] > w ? rowlen[r] : w;
  }
  width[s] = w;
}
#endif

// Exclusive scan of 32 * width into off (one block; chunked sequential scan);
// total[0] = stored entries, total[1] = largest width.
#ifndef AMPCG_INSTANTIATION_UNIT
__global__ void k_slice_offsets(int64_t nslices, const int* width, long long* off,
                                long long* total) {
  __shared__ long long sh[1024];
  __shared__ int shw[1024];
  int t = threadIdx.x, T = blockDim.x;
  int64_t chunk = (nslices + T - 1) / T;
  int64_t a = t * chunk, b = a + chunk < nslices ? a + chunk : nslices;
  long long s = 0;
  int wmax = 0;
  for (int64_t i = a; i < b; ++i) {
    s += 32ll * width[i];
    wmax = width[i] > wmax ? width[i] : wmax;
  }
  sh[t] = s;
  shw[t] = wmax;
  __syncthreads();
  if (t == 0) {
    long long run = 0;
    int m = 0;
    for (int j = 0; j < T; ++j) {
      long long v = sh[j];
      sh[j] = run;
      run += v;
      m = shw[j] > m ? shw[j] : m;
    }
    total[0] = run;
    total[1] = m;
  }
  __syncthreads();
  long long run = sh[t];
  for (int64_t i = a; i < b; ++i) { off[i] = run; run += 32ll * width[i]; }
}
#endif

// Slice-uniform offset patterns (int16 layout): a slice whose 32 rows (all
// below n) have entries only at the offsets of one sorted set U with |U| equal
// to the slice width, every r + u a valid column, is stored with entry j of
// every row at offset U[j] (value 0 where the row has no entry there: the
// row's products and their order are unchanged, the added terms are exact
// zeros).  Its gathers then need U only (one 16-byte pattern per slice), not
// the slice's offsets.  7-point stencils: every slice but the first and the
// last.  One thread per slice.
#ifndef AMPCG_INSTANTIATION_UNIT
__global__ void k_slice_pattern(int64_t n, int64_t nslices, const int* rowptr, const int* col,
                                const int* width, short* pat) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nslices) return;
  const int w = width[s];
  int u[kStageW];
  int m = 0;
  bool ok = w >= 1 && w <= kStageW && s * 32 + 32 <= n;
  for (int l = 0; l < 32 && ok; ++l) {
    const int64_t r = s * 32 + l;
    for (int e = rowptr[r]; e < rowptr[r + 1] && ok; ++e) {
      const int o = col[e] - (int)r;
      int i = 0;
      while (i < m && u[i] < o) ++i;
      if (i < m && u[i] == o) continue;
      if (m == w) { ok = false; break; }
      for (int k = m; k > i; --k) u[k] = u[k - 1];
      u[i] = o;
      ++m;
    }
  }
  ok = ok && m == w;
  for (int i = 0; i < m && ok; ++i) {
    const int64_t lo = s * 32 + u[i], hi = s * 32 + 31 + u[i];
    ok = lo >= 0 && hi < n && u[i] >= -32767 && u[i] <= 32767;
  }
  for (int j = 0; j < kStageW; ++j) pat[s * kStageW + j] = (ok && j < m) ? (short)u[j] : (short)0;
  if (!ok) pat[s * kStageW] = kNoPat;
}
#endif

#ifndef AMPCG_INSTANTIATION_UNIT
__global__ void k_fill_sell(int64_t n, const int* rowptr, const int* col, const double* val,
                            const long long* off, const int* width, const short* pat, int* cabs,
                            short* coff, double* v64, float* v32, unsigned char* rmask) {
  int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t s = row >> 5;
  int lane = (int)(row & 31);
  if (s * 32 >= n) return;
  int w = width[s];
  long long base = off[s] + lane;
  int a = 0, len = 0;
  if (row < n) { a = rowptr[row]; len = rowptr[row + 1] - a; }
  if (pat && pat[s * kStageW] != kNoPat) {
    // uniform slice (every row < n): entry j at offset pat[j], merged with the
    // row's sorted entries
    int e = 0;
    unsigned mk = 0u;
    for (int j = 0; j < w; ++j) {
      const int o = pat[s * kStageW + j];
      double v = 0.0;
      if (e < len && col[a + e] - (int)row == o) {
        v = val[a + (e++)];
        mk |= 1u << j;
      }
      const long long q = base + 32ll * j;
      coff[q] = (short)o;
      v64[q] = v;
      v32[q] = __double2float_rn(v);
    }
    rmask[row] = (unsigned char)mk;
    return;
  }
  for (int j = 0; j < w; ++j) {
    long long e = base + 32ll * j;
    int c = (int)(row < n ? row : 0);
    double v = 0.0;
    if (j < len) { c = col[a + j]; v = val[a + j]; }
    if (cabs) cabs[e] = c;
    if (coff) coff[e] = (short)(row < n ? c - (int)row : 0);
    v64[e] = v;
    v32[e] = __double2float_rn(v);
  }
}
#endif

#ifndef AMPCG_INSTANTIATION_UNIT
__global__ void k_jacobi(int64_t n, const double* diag, double* d64, float* d32, __half* d16) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = 1.0 / diag[i];
  d64[i] = v;
  d32[i] = __double2float_rn(v);
  d16[i] = d2h(v);
}
#endif

// Block CSR (nb block rows of bs x bs blocks, row-major blocks, ascending
// block columns) expanded to scalar CSR: scalar row I*bs + r holds, for each
// block k of block row I, the bs entries of the block's row r.
#ifndef AMPCG_INSTANTIATION_UNIT
__global__ void k_bsr_expand(int64_t nb, int bs, const int* browptr, const int* bcol,
                             const double* bval, int* rowptr, int* col, double* val) {
  int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nb * bs) return;
  int64_t I = row / bs;
  int r = (int)(row % bs);
  int k0 = browptr[I], k1 = browptr[I + 1];
  int64_t start = (int64_t)k0 * bs * bs + (int64_t)r * (k1 - k0) * bs;
  rowptr[row] = (int)start;
  if (row == nb * bs - 1) rowptr[row + 1] = browptr[nb] * bs * bs;
  int64_t o = start;
  for (int k = k0; k < k1; ++k) {
    int J = bcol[k];
    for (int c = 0; c < bs; ++c) {
      col[o] = J * bs + c;
      val[o] = bval[(int64_t)k * bs * bs + (int64_t)r * bs + c];
      ++o;
    }
  }
}
#endif

// New values on the same pattern: vals in CSR order (rowptr on the device),
// written into the sliced layout (FP64 and FP32 copies) with the Jacobi
// inverse diagonal.  flags bit 2: diagonal <= 0; bit 3: non-finite value.
template <int IT>
__global__ void k_update_vals(Sell A, const int* rowptr, const double* vals, double* v64, float* v32,
                              double* d64, float* d32, __half* d16, int* flags) {
  int lane = threadIdx.x & 31;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int s = warp; s < A.nslices; s += nwarps) {
    int row = s * 32 + lane;
    if (row >= A.n) continue;
    long long base = A.off[s] + lane;
    int a = rowptr[row], len = rowptr[row + 1] - a;
    double dg = 0.0;
    int f = 0;
    // entry j of the row holds CSR entry j, or (uniform slices) the next CSR
    // entry when bit j of the row's mask is set
    const bool uni = slice_uniform(A, s);
    const unsigned mk = uni ? A.rmask[row] : 0u;
    const int w = uni ? A.width[s] : len;
    for (int j = 0, k = 0; j < w; ++j) {
      if (uni && !((mk >> j) & 1u)) continue;
      long long e = base + 32ll * j;
      double v = vals[a + (k++)];
      if (!isfinite(v)) f |= 8;
      v64[e] = v;
      v32[e] = __double2float_rn(v);
      if (col_at<IT>(A, e, row) == row) dg = v;
    }
    if (!(dg > 0.0)) f |= 4;
    if (f) atomicOr(flags, f);
    double di = 1.0 / dg;
    d64[row] = di;
    d32[row] = __double2float_rn(di);
    d16[row] = d2h(di);
  }
}

// dL/dA on the pattern (adjoint of A x = b): dLdA[rowptr[i] + j] = -lambda_i x_c
// for the j-th stored entry (column c) of row i, in the caller's CSR order.
template <int IT>
__global__ void k_grad_pattern(Sell A, const int* rowptr, const double* lam, const double* x,
                               double* dLdA) {
  int lane = threadIdx.x & 31;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int s = warp; s < A.nslices; s += nwarps) {
    int row = s * 32 + lane;
    if (row >= A.n) continue;
    long long base = A.off[s] + lane;
    int a = rowptr[row], len = rowptr[row + 1] - a;
    double li = lam[row];
    const bool uni = slice_uniform(A, s);
    const unsigned mk = uni ? A.rmask[row] : 0u;
    const int w = uni ? A.width[s] : len;
    for (int j = 0, k = 0; j < w; ++j) {
      if (uni && !((mk >> j) & 1u)) continue;
      int c = col_at<IT>(A, base + 32ll * j, row);
      dLdA[a + (k++)] = -(li * x[c]);
    }
  }
}

// Log-coefficient field on the matrix graph:
//   a_ij = -exp((theta_i + theta_j)/2) for each stored off-diagonal (i, j),
//   a_ii = sum_{j != i} exp((theta_i + theta_j)/2) + nb_i exp(theta_i)
// (nb_i = number of boundary faces of node i).  Writes the FP64/FP32 copies
// and the Jacobi inverse diagonal.  flags bit 2: no stored diagonal.
template <int IT>
__global__ void k_assemble_logcoeff(Sell A, const double* theta, const int* nb, double* v64,
                                    float* v32, double* d64, float* d32, __half* d16, int* flags) {
  int lane = threadIdx.x & 31;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int s = warp; s < A.nslices; s += nwarps) {
    int row = s * 32 + lane;
    if (row >= A.n) continue;
    long long base = A.off[s] + lane;
    int w = A.width[s];
    double ti = theta[row], sum = 0.0;
    long long ed = -1;
    const bool uni = slice_uniform(A, s);
    const unsigned mk = uni ? A.rmask[row] : 0u;
    for (int j = 0; j < w; ++j) {
      if (uni && !((mk >> j) & 1u)) continue;   // an added zero stays zero
      long long e = base + 32ll * j;
      int c = col_at<IT>(A, e, row);
      if (c == row) {
        if (ed < 0) ed = e;   // padding repeats (0, row) after the real entries
        continue;
      }
      double kf = exp(0.5 * (ti + theta[c]));
      sum += kf;
      v64[e] = -kf;
      v32[e] = __double2float_rn(-kf);
    }
    if (ed < 0) { atomicOr(flags, 4); continue; }
    double dg = sum + (double)nb[row] * exp(ti);
    v64[ed] = dg;
    v32[ed] = __double2float_rn(dg);
    double di = 1.0 / dg;
    d64[row] = di;
    d32[row] = __double2float_rn(di);
    d16[row] = d2h(di);
  }
}

// dL/dtheta for the log-coefficient field, from the forward solution x and
// the adjoint lambda (A lambda = dL/dx): with dL/da_ij = -lambda_i x_j,
//   dL/dtheta_i = sum_{j != i} -(lambda_i - lambda_j)(x_i - x_j) k_ij / 2
//                 - lambda_i x_i kb_i,
// k_ij = -a_ij and kb_i = nb_i exp(theta_i) = sum_j a_ij (the row sum).
// One thread per row, ascending column order: deterministic.
template <int IT>
__global__ void k_grad_logcoeff(Sell A, const double* x, const double* lam, double* dtheta) {
  int lane = threadIdx.x & 31;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int s = warp; s < A.nslices; s += nwarps) {
    int row = s * 32 + lane;
    if (row >= A.n) continue;
    long long base = A.off[s] + lane;
    int w = A.width[s];
    double xi = x[row], li = lam[row], g = 0.0, rowsum = 0.0;
    bool seen_diag = false;
    const bool uni = slice_uniform(A, s);
    const unsigned mk = uni ? A.rmask[row] : 0u;
    for (int j = 0; j < w; ++j) {
      if (uni && !((mk >> j) & 1u)) continue;
      long long e = base + 32ll * j;
      int c = col_at<IT>(A, e, row);
      double a = A.v64[e];
      if (c == row) {
        if (!seen_diag) rowsum += a;   // padding repeats (0, row)
        seen_diag = true;
        continue;
      }
      rowsum += a;
      g += -((li - lam[c]) * (xi - x[c])) * (-a) * 0.5;
    }
    dtheta[row] = g - li * xi * rowsum;
  }
}


// ---------------------------------------------------------------------------
// Chebyshev polynomial preconditioner (reading R8): M^-1 = D^-1/2 P(Ahat)
// D^-1/2, Ahat = D^-1/2 A D^-1/2, applied as m steps of the Chebyshev
// iteration for Ahat u = v (Saad, Iterative Methods for Sparse Linear
// Systems, Alg. 12.1) from u_0 = 0 on [lmin, lmax]:
//   v = D^-1/2 y, res = v, d_0 = v / theta, u = d_0;
//   step j = 1..m-1: t = Ahat d_{j-1}; res -= t;
//                    d_j = c1_j d_{j-1} + c2_j res; u += d_j;
//   z = D^-1/2 u.
// All vectors in u_z (FP16/FP32 ones computed in FP32 and rounded once); the
// product uses the copy of Ahat in u_z.  c1_j, c2_j, 1/theta are FP64
// constants computed once on the host.
struct Cheb {
  const double* ah64;
  const float* ah32;
  const __half* ah16;
  // binary16 Ahat value and int16 column offset of each stored entry in one
  // 32-bit word (value in the low half), when the offsets fit: one load per
  // entry instead of two for the FP16 steps
  const unsigned* ahp;
  const double* ds64;
  const float* ds32;
  const __half* ds16;
  void* res;
  void* d[2];
  void* u;
  double inv_theta;
};

template <int UZ> __device__ __forceinline__ typename Store<UZ>::T cheb_ds(const Cheb& C, int64_t i);
template <> __device__ __forceinline__ double cheb_ds<P64>(const Cheb& C, int64_t i) { return C.ds64[i]; }
template <> __device__ __forceinline__ float cheb_ds<P32>(const Cheb& C, int64_t i) { return C.ds32[i]; }
template <> __device__ __forceinline__ __half cheb_ds<P16>(const Cheb& C, int64_t i) { return C.ds16[i]; }

// a * b in u_z: FP64 multiply, or the FP32 product rounded once.
template <int UZ>
__device__ __forceinline__ typename Store<UZ>::T mul_u(typename Store<UZ>::T a, typename Store<UZ>::T b) {
  if constexpr (UZ == P64) return __dmul_rn(a, b);
  else if constexpr (UZ == P32) return __fmul_rn(a, b);
  else return __float2half_rn(__fmul_rn(__half2float(a), __half2float(b)));
}
template <int UZ>
__device__ __forceinline__ typename Store<UZ>::T add_u(typename Store<UZ>::T a, typename Store<UZ>::T b) {
  if constexpr (UZ == P64) return __dadd_rn(a, b);
  else if constexpr (UZ == P32) return __fadd_rn(a, b);
  else return __float2half_rn(__fadd_rn(__half2float(a), __half2float(b)));
}
template <int UZ>
__device__ __forceinline__ typename Store<UZ>::T sub_u(typename Store<UZ>::T a, typename Store<UZ>::T b) {
  if constexpr (UZ == P64) return __dsub_rn(a, b);
  else if constexpr (UZ == P32) return __fsub_rn(a, b);
  else return __float2half_rn(__fsub_rn(__half2float(a), __half2float(b)));
}

// y = omega r (as in precond_rows), v = D^-1/2 y, res = v, d_0 = v/theta, u = d_0.
template <int UZ, int UR>
__global__ void __launch_bounds__(256) k_cheb_init(Bufs B, Cheb C, int64_t n, DevState* st) {
  using TZ = typename Store<UZ>::T;
  using TR = typename Store<UR>::T;
  __shared__ DevState S;
  if (!state_enter(&S, st, UZ, UR)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) st->phase_runs[2 * UZ + UR] += 1;
  const int r_cast = S.r_cast;
  const double om = S.omega;
  const float omf = S.omega_f;
  const int pow2 = S.omega_pow2, oe = S.omega_e;
  const bool om_one = pow2 && oe == 0;
  TZ* res = (TZ*)C.res;
  TZ* d0 = (TZ*)C.d[0];
  TZ* u = (TZ*)C.u;
  TZ it;
  if constexpr (UZ == P64) it = C.inv_theta;
  else if constexpr (UZ == P32) it = __double2float_rn(C.inv_theta);
  else it = __float2half_rn(__double2float_rn(C.inv_theta));   // unused for FP16 (FP32 constant below)
  const float itf = __double2float_rn(C.inv_theta);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    TR r;
    if constexpr (UR == P64) {
      if (r_cast) { r = f2d(B.r32[i]); B.r64[i] = r; } else r = B.r64[i];
    } else {
      if (r_cast) { r = __double2float_rn(B.r64[i]); B.r32[i] = r; } else r = B.r32[i];
    }
    TZ y;
    if constexpr (UR == P64) {
      if constexpr (UZ == P16) y = pow2 ? d2h_scaled(r, oe) : d2h(__dmul_rn(om, r));
      else y = round_from_f64<UZ>(om_one ? r : __dmul_rn(om, r));
    } else {
      y = round_from_f32<UZ>(__fmul_rn(omf, r));
    }
    TZ v = mul_u<UZ>(cheb_ds<UZ>(C, i), y);
    TZ dd;
    if constexpr (UZ == P64) dd = __dmul_rn(v, it);
    else if constexpr (UZ == P32) dd = __fmul_rn(v, itf);
    else dd = __float2half_rn(__fmul_rn(__half2float(v), itf));
    res[i] = v;
    d0[i] = dd;
    u[i] = dd;
  }
  if (S.p_cast) cast_p<UZ>(B, n, &S);
}

// One Chebyshev step j >= 1: t = Ahat d_{j-1} (accumulated in u_z's compute
// precision), res -= t, d_j = c1 d_{j-1} + c2 res, u += d_j.  Thread per row.
// Row product of the packed FP16 Chebyshev matrix (Cheb::ahp): FP32
// accumulation in ascending entry order, 8 entries per chunk with the next
// chunk's words loaded before the current chunk's gathers.
__device__ __forceinline__ float row_sum_packed16(const unsigned* __restrict__ ahp, long long base, int w,
                                                  int row, const __half* __restrict__ x) {
  constexpr int CH = 8;
  unsigned a[CH];
#pragma unroll
  for (int u = 0; u < CH; ++u) a[u] = (u < w) ? __ldg(ahp + base + 32 * u) : 0u;
  float acc = 0.f;
  for (int j0 = 0; j0 < w; j0 += CH) {
    unsigned an[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int j = j0 + CH + u;
      an[u] = (j < w) ? __ldg(ahp + base + 32 * j) : 0u;
    }
    __half g[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u)
      if (j0 + u < w) g[u] = x[row + (int)(short)(a[u] >> 16)];
#pragma unroll
    for (int u = 0; u < CH; ++u)
      if (j0 + u < w)
        acc = __fmaf_rn(__half2float(__ushort_as_half((unsigned short)(a[u] & 0xffffu))), __half2float(g[u]), acc);
#pragma unroll
    for (int u = 0; u < CH; ++u) a[u] = an[u];
  }
  return acc;
}

template <int UZ, int UR, int IT>
__global__ void __launch_bounds__(256) k_cheb_step(Sell A, Cheb C, DevState* st, int j, double c1,
                                                   double c2) {
  using TZ = typename Store<UZ>::T;
  {
    // one round of loads for the entry test (no other state is read)
    const int dn = st->done, uz = st->uz, ur = st->ur;
    if (dn || uz != UZ || ur != UR) return;
  }
  const TZ* __restrict__ dp = (const TZ*)(((j - 1) & 1) ? C.d[1] : C.d[0]);
  TZ* dn = (TZ*)((j & 1) ? C.d[1] : C.d[0]);
  TZ* res = (TZ*)C.res;
  TZ* u = (TZ*)C.u;
  const float c1f = __double2float_rn(c1), c2f = __double2float_rn(c2);
  int lane = threadIdx.x & 31;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int s = warp; s < A.nslices; s += nwarps) {
    int row = s * 32 + lane;
    if (row >= A.n) continue;
    long long base = __ldg(A.off + s) + lane;
    int w = __ldg(A.width + s);
    TZ t;
    if constexpr (UZ == P64) {
      t = row_sum_chunked<IT>(A, C.ah64, base, w, row, 0.0, [=](int j) { return dp[j]; },
                              [](double av, double xv, double s) { return fma(av, xv, s); });
    } else if constexpr (UZ == P32) {
      t = row_sum_chunked<IT>(A, C.ah32, base, w, row, 0.f, [=](int j) { return dp[j]; },
                              [](float av, float xv, float s) { return __fmaf_rn(av, xv, s); });
    } else {
      float acc;
      if (IT == 1 && C.ahp) {
        acc = row_sum_packed16(C.ahp, base, w, row, dp);
      } else {
        acc = row_sum_chunked<IT>(A, C.ah16, base, w, row, 0.f, [=](int j) { return dp[j]; },
                                  [](__half av, __half xv, float s) {
                                    return __fmaf_rn(__half2float(av), __half2float(xv), s);
                                  });
      }
      t = __float2half_rn(acc);
    }
    TZ rs = sub_u<UZ>(res[row], t);
    TZ dd;
    if constexpr (UZ == P64) dd = fma(c1, dp[row], __dmul_rn(c2, rs));
    else if constexpr (UZ == P32) dd = __fmaf_rn(c1f, dp[row], __fmul_rn(c2f, rs));
    else dd = __float2half_rn(__fmaf_rn(c1f, __half2float(dp[row]), __fmul_rn(c2f, __half2float(rs))));
    res[row] = rs;
    dn[row] = dd;
    u[row] = add_u<UZ>(u[row], dd);
  }
}

// z = D^-1/2 u, rho = r^T z (as k_precond), last block: beta.
template <int UZ, int UR>
__global__ void __launch_bounds__(256) k_cheb_final(Bufs B, Cheb C, int64_t n, DevState* st) {
  using TZ = typename Store<UZ>::T;
  using TR = typename Store<UR>::T;
  __shared__ DevState S;
  if (!state_enter(&S, st, UZ, UR)) return;
  constexpr bool kSmall = (UR != P64) && (UZ != P64);
  const TZ* u = (const TZ*)C.u;
  TZ* z = (TZ*)B.z;
  const float sigf = S.sig_f;
  double rho = 0.0;
  Dot2 d2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    TZ zi = mul_u<UZ>(cheb_ds<UZ>(C, i), u[i]);
    z[i] = zi;
    TR r;
    if constexpr (UR == P64) r = B.r64[i];
    else r = B.r32[i];
    if constexpr (kSmall) d2.add(__fmul_rn((float)r, sigf), (float)zi);
    else rho = fma(to_f64(r), to_f64(zi), rho);
  }
  double v[1];
  if constexpr (kSmall) {
    v[0] = block_sum_dot2(d2, S.inv_sig);
  } else {
    v[0] = rho;
    block_sum<1>(v);
  }
  if (threadIdx.x == 0) B.part[blockIdx.x] = v[0];
  if (!last_block(&st->ticket[0])) return;
  state_load(&S, st);
  double tot[1];
  final_sum<1>(B.part, gridDim.x, 1, tot);
  if (threadIdx.x == 0) {
    S.ticket[0] = 0u;
    rho_step(&S, tot[0]);
    if (S.redo) {   // the lagged scale is not offered with Chebyshev (the host rejects it)
      S.redo = 0;
      S.status = ST_NONFINITE;
      S.done = 1;
    }
  }
  state_store(st, &S);
}

// Ahat = D^-1/2 A D^-1/2 in the sliced layout ((dsi_i a_ij) dsi_j in FP64,
// rounded to FP32/FP16), D^-1/2 in three precisions, and the Gershgorin bound
// max_i sum_j |ahat_ij| (as an order-preserving key) for the interval.
template <int IT>
__global__ void k_cheb_setup(Sell A, double* ah64, float* ah32, __half* ah16, double* ds64,
                             float* ds32, __half* ds16, unsigned long long* gersh) {
  int lane = threadIdx.x & 31;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int nwarps = (gridDim.x * blockDim.x) >> 5;
  // pass 1: D^-1/2
  for (int s = warp; s < A.nslices; s += nwarps) {
    int row = s * 32 + lane;
    if (row >= A.n) continue;
    long long base = A.off[s] + lane;
    int w = A.width[s];
    double dg = 0.0;
    for (int j = 0; j < w; ++j) {
      long long e = base + 32ll * j;
      if (col_at<IT>(A, e, row) == row) { dg = A.v64[e]; break; }
    }
    double di = 1.0 / sqrt(dg);
    ds64[row] = di;
    ds32[row] = __double2float_rn(di);
    ds16[row] = d2h(di);
  }
}

template <int IT>
__global__ void k_cheb_setup2(Sell A, const double* ds64, double* ah64, float* ah32, __half* ah16,
                              unsigned* ahp, unsigned long long* gersh) {
  int lane = threadIdx.x & 31;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int s = warp; s < A.nslices; s += nwarps) {
    int row = s * 32 + lane;
    if (row >= A.n) continue;
    long long base = A.off[s] + lane;
    int w = A.width[s];
    double di = ds64[row], sum = 0.0;
    for (int j = 0; j < w; ++j) {
      long long e = base + 32ll * j;
      int c = col_at<IT>(A, e, row);
      double ah = __dmul_rn(__dmul_rn(di, A.v64[e]), ds64[c]);
      ah64[e] = ah;
      ah32[e] = __double2float_rn(ah);
      const __half h = d2h(ah);
      ah16[e] = h;
      if (IT == 1 && ahp)
        ahp[e] = ((unsigned)(unsigned short)A.coff[e] << 16) | (unsigned)__half_as_ushort(h);
      sum += fabs(ah);
    }
    atomicMax(gersh, abs_key(sum));
  }
}

// ---------------------------------------------------------------------------
// Step entry points (single launches, no reduction).

template <int UR, int IT>
__global__ void __launch_bounds__(256) k_spmv_step(Sell A, const void* p, void* q) {
  using TR = typename Store<UR>::T;
  int lane = threadIdx.x & 31;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int s = warp; s < A.nslices; s += nwarps) {
    int row = s * 32 + lane;
    if (row < A.n) ((TR*)q)[row] = sell_row<UR, UR, IT>(A, s, lane, row, (const TR*)p);
  }
}

template <int IT>
__global__ void __launch_bounds__(256) k_residual_step(Sell A, const double* b, const double* x,
                                                       double* r) {
  int lane = threadIdx.x & 31;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int s = warp; s < A.nslices; s += nwarps) {
    int row = s * 32 + lane;
    if (row < A.n) r[row] = b[row] - sell_row64<IT>(A, s, lane, row, x);
  }
}

// z = M^-1 round_uz(omega r): the same row arithmetic as k_precond, without
// the reduction, on caller arrays.  The state block carries omega.
template <int UZ, int UR, int MT>
__global__ void __launch_bounds__(256) k_precond_step(Bufs B, int64_t n, const DevState* st) {
  double rho = 0.0;
  Dot2 d2;
  precond_rows<UZ, UR, MT, 1>(B, n, st, rho, d2);
}

// Failure-detection check of the grid barrier: a cooperative launch of
// gridDim.x blocks meets at one grid_reduce_barrier with a caller-given poll
// limit; block `absent` (if in range) returns without arriving, so the others'
// wait runs out after `spin` polls and they report it.  out[b] = 1 when block b
// passed the barrier, 0 when its wait ran out, -1 when it did not arrive.
#ifndef AMPCG_INSTANTIATION_UNIT
__global__ void __launch_bounds__(256) k_barrier_check(GridSumBarrier* g, double* part, int absent,
                                                       long long spin, int* out) {
  if ((int)blockIdx.x == absent) {
    if (threadIdx.x == 0) out[blockIdx.x] = -1;
    return;
  }
  int nb = 0;
  double tot = 0.0;
  unsigned long long mtot = 0ull;
  const bool ok = grid_reduce_barrier<1>(g, part, nullptr, nb, 1.0, 0ull, tot, mtot, spin);
  if (threadIdx.x == 0) out[blockIdx.x] = (ok && tot == (double)gridDim.x) ? 1 : 0;
}
#endif

// Selector replay over a residual-norm sequence (one thread).
#ifndef AMPCG_INSTANTIATION_UNIT
__global__ void k_selector_trace(DevState* st, int m, unsigned char* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  prep_selector(st);
  for (int k = 0; k <= m; ++k) {
    st->k = k;
    st->delta = st->delta_hist[k];
    decide(st, ArrayHist{st->delta_hist});
    out[k] = st->prec_hist[k];
    st->first = 0;
  }
}
#endif

}  // namespace ampcg
