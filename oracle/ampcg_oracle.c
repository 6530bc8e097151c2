/*
 * ampcg_oracle.c -- plain, slow CPU oracle for AMP-PCG / DS-PCG.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant generator
 * with the CUDA library.
 *
 * What it computes (Guo, de Sturler, Warburton, "An Adaptive Mixed-Precision
 * and Dynamically Scaled Preconditioned Conjugate Gradient Algorithm"):
 *   - PCG, Algorithm 1, in native FP64                          (oracle_pcg64)
 *   - DS-PCG, Algorithm 2, and AMP-PCG, Algorithm 3, with every vector
 *     stored through a software rounding to the precision the paper assigns
 *     to it (Sec. 4: u_r for y-compute, q and r; u_z for y-store, z and p;
 *     x, inner products, norms and scalars in FP64)               (oracle_ampcg)
 *   - the precision selector of Eq. (precision_selector)     (oracle_select)
 *   - the attainable-accuracy indicators: the delay-window form, Eq. (eta_k),
 *     and the linear-convergence form, Eq. (linear criterion)    (oracle_eta_*)
 *   - the a-posteriori indicator hat-eta_m(k) of Eq. (Weta_k)  (oracle_eta_hat)
 *
 * Readings where the paper is silent (numbered as in the design notes):
 *   R1  eps32 = 2^-24 (unit roundoff of binary32).
 *   R2  u_r switches to FP32 iff eta_k <= tol*||b||  (the criterion equation;
 *       the selector's "eta_k < tol" is read as the same absolute test).
 *   R3  no u_r switch before k >= d (window) or k >= ell (linear); inside the
 *       window ||r_{-1}|| := ||r_0||.
 *   R4  latch: a precision never rises again within a solve (flag).
 *   R5  scale modes: NONE (omega=1), L2 (omega = 1/delta_k as in Alg. 3),
 *       LINF_POW2 (omega = 2^-ceil(log2 max|r_k|), an exact power of two;
 *       Sec. 3.3 allows any nonzero omega).
 *       LINF_POW2_LAG: the same power of two taken from the previous
 *       iteration's residual, omega_k = 2^-ceil(log2 max|r_{k-1}|) for k >= 1
 *       (omega_0 from r_0); Sec. 3.3 names a lagged factor (1/||z_{k-1}||)
 *       as a practical choice.  If rho_k comes out non-finite (y overflowed
 *       u_z because r grew), y_k, z_k and rho_k are formed once more with
 *       omega_k = 2^-ceil(log2 max|r_k|)                        (R20)
 *   R6  y_i = round_uz( fl_ur(omega * r_i) ): one multiply, computed in u_r,
 *       stored in u_z.
 *   R7  FP16 quantities are computed in FP32 (with fma where the formula is a
 *       multiply-add) and rounded once to FP16; FP32 quantities in FP32; the
 *       SpMV uses the copy of A in u_r and accumulates in u_r, ascending
 *       column order, one fma per nonzero.
 *   R9  optional true-residual refresh after convergence of the updated
 *       residual (verify_refresh).
 *   R10 at a u_r switch r_k is rounded once to FP32 before y_k is formed.
 *   R12 rho <= 0, gamma <= 0 -> breakdown; non-finite scalars -> nonfinite.
 *   Inner products are plain recursive sums in FP64 in ascending index order
 *   (s = s + a_i*b_i, products rounded to FP64, no fma contraction).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_FP64 0
#define OR_FP32 1
#define OR_FP16 2

#define OR_CRIT_WINDOW 0
#define OR_CRIT_LINEAR 1
#define OR_CRIT_FIXED 2

#define OR_SCALE_NONE 0
#define OR_SCALE_L2 1
#define OR_SCALE_LINF_POW2 2
#define OR_SCALE_LINF_POW2_LAG 3

#define OR_M_NONE 0
#define OR_M_JACOBI 1
#define OR_M_CHEBYSHEV 2

#define OR_OK 0
#define OR_NOT_CONVERGED 1
#define OR_ERR_INVALID (-1)
#define OR_ERR_BREAKDOWN (-3)
#define OR_ERR_NONFINITE (-4)

/* R1: unit roundoff of binary32. */
static const double EPS32 = 5.9604644775390625e-08; /* 2^-24 */

/* ------------------------------------------------------------------------ */
/* IEEE 754 round-to-nearest-even into a binary format with `p` significand
 * bits (including the hidden bit) and minimum normal exponent `emin`,
 * maximum exponent `emax`.  Written from the definition: the representable
 * numbers in the binade [2^e, 2^(e+1)) are multiples of 2^(e-p+1); below
 * 2^emin the spacing stays 2^(emin-p+1) (subnormals); a result whose
 * magnitude rounds to 2^(emax+1) or above overflows to infinity.           */
static double round_to_format(double v, int p, int emin, int emax) {
  if (isnan(v) || isinf(v) || v == 0.0) return v;
  double a = fabs(v);
  int E;
  (void)frexp(a, &E); /* a = f * 2^E, f in [0.5, 1): floor(log2 a) = E-1 */
  int e = E - 1;
  if (e < emin) e = emin;
  double quantum = ldexp(1.0, e - p + 1);
  double t = a / quantum;      /* exact: scaling by a power of two */
  double n = nearbyint(t);     /* round half to even (default mode) */
  double res = n * quantum;    /* exact */
  double maxfin = ldexp(2.0 - ldexp(1.0, 1 - p), emax);
  if (res > maxfin) res = INFINITY;
  return copysign(res, v);
}

double oracle_round16(double v) { return round_to_format(v, 11, -14, 15); }
double oracle_round32(double v) { return round_to_format(v, 24, -126, 127); }

double oracle_round(int prec, double v) {
  if (prec == OR_FP16) return oracle_round16(v);
  if (prec == OR_FP32) return oracle_round32(v);
  return v;
}

void oracle_round_array(int prec, const double* in, double* out, int64_t n) {
  for (int64_t i = 0; i < n; ++i) out[i] = oracle_round(prec, in[i]);
}

/* Binary32 arithmetic on values that are already binary32-representable:
 * the host FPU's float ops are IEEE binary32 ops (x86-64 SSE, no excess
 * precision), fmaf is the correctly rounded fused multiply-add. */
static double mul32(double a, double b) { return (double)((float)a * (float)b); }
static double fma32(double a, double b, double c) {
  return (double)fmaf((float)a, (float)b, (float)c);
}

/* ------------------------------------------------------------------------ */
/* Sparse kernels.  CSR with ascending column indices in each row.          */

/* q = A p in precision `prec` (R7): FP64: fma chain in FP64; FP32: fma chain
 * in FP32 over the FP32 copy of A and p rounded to FP32; FP16: fma chain in
 * FP32 over the FP16 copy of A and p rounded to FP16, result rounded once to
 * FP16.  `aval` holds the matrix copy already rounded to `prec`.           */
void oracle_spmv(int64_t n, const int32_t* rowptr, const int32_t* col,
                 const double* aval, int prec, const double* p, double* q) {
  for (int64_t i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      double pj = p[col[k]];
      if (prec == OR_FP64) {
        acc = fma(aval[k], pj, acc);
      } else {
        double pr = oracle_round(prec, pj);
        acc = fma32(aval[k], pr, acc);
      }
    }
    q[i] = oracle_round(prec, acc);
  }
}

/* r = b - A x in FP64 (Alg. 3 initial residual): t_i = sum_j a_ij x_j as an FP64 fma
 * chain in ascending column order, then r_i = b_i - t_i.                   */
void oracle_residual64(int64_t n, const int32_t* rowptr, const int32_t* col,
                       const double* val, const double* b, const double* x,
                       double* r) {
  for (int64_t i = 0; i < n; ++i) {
    double t = 0.0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) t = fma(val[k], x[col[k]], t);
    r[i] = b[i] - t;
  }
}

/* Plain FP64 inner product, ascending order, products rounded then added.  */
double oracle_dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double prod = a[i] * b[i];
    s = s + prod;
  }
  return s;
}

double oracle_nrm2(int64_t n, const double* a) { return sqrt(oracle_dot(n, a, a)); }

double oracle_maxabs(int64_t n, const double* a) {
  double m = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double v = fabs(a[i]);
    if (v > m) m = v;
  }
  return m;
}

/* Diagonal of a CSR matrix (0 where absent). */
static void csr_diag(int64_t n, const int32_t* rowptr, const int32_t* col,
                     const double* val, double* d) {
  for (int64_t i = 0; i < n; ++i) {
    d[i] = 0.0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (col[k] == i) d[i] = val[k];
  }
}

/* ------------------------------------------------------------------------ */
/* Scale factor omega_k (R5).  LINF_POW2: with m = max|r_k| = f*2^E,
 * f in [0.5,1): ceil(log2 m) = E-1 if f == 0.5 else E; omega = 2^-ceil(.),
 * so max|omega r| lies in (0.5, 1].                                        */
double oracle_scale(int mode, double delta, double maxabs) {
  if (mode == OR_SCALE_L2) return 1.0 / delta;
  if (mode == OR_SCALE_LINF_POW2 || mode == OR_SCALE_LINF_POW2_LAG) {
    if (!(maxabs > 0.0) || isinf(maxabs)) return 1.0;
    int E;
    double f = frexp(maxabs, &E);
    int c = (f == 0.5) ? E - 1 : E;
    return ldexp(1.0, -c);
  }
  return 1.0;
}

/* ------------------------------------------------------------------------ */
/* Attainable-accuracy indicators.  delta[t] = ||r_t||, t = 0..k.          */

/* Delay-window form, Eq. (eta_k):
 *   eta_k = sum_{t=k-d}^{k} eps32 ( (3+C) ||r_{t-1}|| + (2+C) ||r_t|| ),
 * with R3: +inf for k < d, ||r_{-1}|| := ||r_0||.                          */
double oracle_eta_window(const double* delta, int k, int d, double C) {
  if (k < d) return INFINITY;
  double eta = 0.0;
  for (int t = k - d; t <= k; ++t) {
    double prev = (t >= 1) ? delta[t - 1] : delta[0];
    double term = EPS32 * ((3.0 + C) * prev + (2.0 + C) * delta[t]);
    eta = eta + term;
  }
  return eta;
}

/* Linear-convergence form, Eq. (linear criterion):
 *   rho = (||r_k|| / ||r_{k-ell}||)^(1/ell),
 *   eta_k = eps32 (5+2C) ||r_{k-1}|| / (1 - rho),
 * with R3 (+inf for k < ell) and +inf when rho >= 1.                      */
double oracle_eta_linear(const double* delta, int k, int ell, double C) {
  if (k < ell || k < 1) return INFINITY;
  double rho = pow(delta[k] / delta[k - ell], 1.0 / (double)ell);
  if (!(rho < 1.0)) return INFINITY;
  return EPS32 * (5.0 + 2.0 * C) * delta[k - 1] / (1.0 - rho);
}

/* A-posteriori indicator hat-eta_m(k), Eq. (Weta_k): FP64 roundoff before
 * the switch at k, FP32 after it, summed over t = 0..m.  Diagnostic only.   */
double oracle_eta_hat(const double* delta, int k, int m, double C) {
  const double eps64 = 1.1102230246251565e-16; /* 2^-53 */
  double s = 0.0;
  for (int t = 0; t <= m; ++t) {
    double prev = (t >= 1) ? delta[t - 1] : delta[0];
    double w = (3.0 + C) * prev + (2.0 + C) * delta[t];
    if (t <= k) s = s + eps64 * w;
    if (t >= k) s = s + EPS32 * w;
  }
  return s;
}

/* Precision selector, Eq. (precision_selector).  Precisions are ordered
 * FP64 (0) > FP32 (1) > FP16 (2); "min" of two precisions (the lower one)
 * is the larger code.  tol_nb = tol * ||b|| (R2).                         */
void oracle_select(double nu, int u0, double tau_zs, double tau_zh, double eta,
                   double tol_nb, int* uz, int* ur) {
  int z;
  if (nu >= tau_zs) z = u0;
  else if (nu >= tau_zh) z = (u0 > OR_FP32) ? u0 : OR_FP32;
  else z = (u0 > OR_FP16) ? u0 : OR_FP16;
  *uz = z;
  *ur = (eta <= tol_nb) ? OR_FP32 : OR_FP64;
}

/* ------------------------------------------------------------------------ */
typedef struct {
  int u0;          /* initial u_z precision */
  int criterion;   /* OR_CRIT_WINDOW / LINEAR / FIXED */
  int d;           /* window delay (Eq. eta_k) */
  int ell;         /* rate window (Eq. linear criterion) */
  double C;        /* Assumption 1 constant */
  double tau_zs;   /* FP64 -> FP32 threshold for u_z */
  double tau_zh;   /* FP32 -> FP16 threshold for u_z */
  int scale;       /* OR_SCALE_* */
  int latch;       /* R4 */
  int verify_refresh; /* R9: max refreshes (0 = off) */
  int fixed_uz;    /* FIXED criterion: constant u_z */
  int fixed_ur;    /* FIXED criterion: constant u_r (FP16 allowed here) */
} oracle_policy;

typedef struct {
  int status;
  int iters;
  int converged;
  int refreshes;
  double true_relres;
  double updated_relres;
  int switch_iter[3]; /* u_z -> FP32, u_z -> FP16, u_r -> FP32; -1 if none */
  int scale_retries;  /* R20: iterations whose scaling was formed again */
  int64_t y16_small;  /* binary16 y_i below the normal range (subnormal or 0) while r_i != 0 */
  int64_t y16_total;  /* binary16 y_i with r_i != 0 (both summed over the iterations) */
} oracle_result;

/* Chebyshev data for M^-1 = D^-1/2 P(Ahat) D^-1/2 (see oracle_cheb_apply). */
typedef struct {
  int degree;
  double lmin, lmax;          /* interval [a, b] for Ahat */
  const double* ahat[3];      /* Ahat values rounded to FP64/FP32/FP16 */
  const double* dsqrt_inv[3]; /* D^-1/2 rounded to FP64/FP32/FP16 */
} oracle_cheb;

/* Chebyshev preconditioner apply in precision `u` (reading R8): z = D^-1/2
 * u_m with u_m the m-th iterate of the Chebyshev iteration (Saad,
 * Iterative Methods for Sparse Linear Systems, Alg. 12.1) for Ahat u = v,
 * v = D^-1/2 y, started from u_0 = 0 on the interval [lmin, lmax]:
 *   theta = (b+a)/2, delta = (b-a)/2, sigma = theta/delta, rho_0 = 1/sigma,
 *   res_0 = v, d_0 = res_0 / theta,
 *   for j = 0..m-1:  u_{j+1} = u_j + d_j
 *                    (j < m-1) res_{j+1} = res_j - Ahat d_j,
 *                              rho_{j+1} = 1/(2 sigma - rho_j),
 *                              d_{j+1} = rho_{j+1} rho_j d_j
 *                                        + (2 rho_{j+1}/delta) res_{j+1}.
 * Scalars are FP64; vectors are stored in u (FP16 ones computed in FP32 and
 * rounded, R7); the product Ahat d uses the copy of Ahat in u.             */
static void oracle_cheb_apply(int64_t n, const int32_t* rowptr, const int32_t* col,
                              const oracle_cheb* ch, int u, const double* y,
                              double* z, double* wv, double* wres, double* wd,
                              double* wt) {
  const double* ah = ch->ahat[u];
  const double* ds = ch->dsqrt_inv[u];
  double a = ch->lmin, bb = ch->lmax;
  double theta = (bb + a) / 2.0, delt = (bb - a) / 2.0;
  double sigma = theta / delt;
  double rho = 1.0 / sigma;
  int m = ch->degree;
  /* v = D^-1/2 y ; res = v ; d = v/theta ; u = 0 */
  for (int64_t i = 0; i < n; ++i) {
    double v;
    if (u == OR_FP64) v = ds[i] * y[i];
    else v = oracle_round(u, mul32(ds[i], y[i]));
    wres[i] = v;
    if (u == OR_FP64) wd[i] = v * (1.0 / theta);
    else wd[i] = oracle_round(u, mul32(v, oracle_round32(1.0 / theta)));
    wv[i] = 0.0;
  }
  for (int j = 0; j < m; ++j) {
    for (int64_t i = 0; i < n; ++i) {
      if (u == OR_FP64) wv[i] = wv[i] + wd[i];
      else wv[i] = oracle_round(u, (double)((float)wv[i] + (float)wd[i]));
    }
    if (j == m - 1) break;
    /* res = res - Ahat d (SpMV accumulated in u's compute precision) */
    oracle_spmv(n, rowptr, col, ah, u, wd, wt);
    double rho_next = 1.0 / (2.0 * sigma - rho);
    double c1 = rho_next * rho, c2 = 2.0 * rho_next / delt;
    for (int64_t i = 0; i < n; ++i) {
      if (u == OR_FP64) {
        wres[i] = wres[i] - wt[i];
        wd[i] = fma(c1, wd[i], c2 * wres[i]);
      } else {
        wres[i] = oracle_round(u, (double)((float)wres[i] - (float)wt[i]));
        double t2 = mul32(oracle_round32(c2), wres[i]);
        wd[i] = oracle_round(u, fma32(oracle_round32(c1), wd[i], t2));
      }
    }
    rho = rho_next;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (u == OR_FP64) z[i] = ds[i] * wv[i];
    else z[i] = oracle_round(u, mul32(ds[i], wv[i]));
  }
}

/* Public wrapper so tests can check the recurrence against the closed-form
 * polynomial on small matrices.  `ahat64` is Ahat in FP64, `dsi64` the FP64
 * D^-1/2; lower-precision copies are formed here by rounding.              */
int oracle_cheb_apply_public(int64_t n, int64_t nnz, const int32_t* rowptr,
                             const int32_t* col, const double* ahat64,
                             const double* dsi64, int degree, double lmin,
                             double lmax, int u, const double* y, double* z) {
  oracle_cheb ch;
  double* buf = (double*)malloc(sizeof(double) * (size_t)(2 * nnz + 2 * n + 4 * n));
  if (!buf) return OR_ERR_INVALID;
  double* ah32 = buf; double* ah16 = buf + nnz;
  double* ds32 = buf + 2 * nnz; double* ds16 = ds32 + n;
  double* w = ds16 + n;
  for (int64_t k = 0; k < nnz; ++k) { ah32[k] = oracle_round32(ahat64[k]); ah16[k] = oracle_round16(ahat64[k]); }
  for (int64_t i = 0; i < n; ++i) { ds32[i] = oracle_round32(dsi64[i]); ds16[i] = oracle_round16(dsi64[i]); }
  ch.degree = degree; ch.lmin = lmin; ch.lmax = lmax;
  ch.ahat[0] = ahat64; ch.ahat[1] = ah32; ch.ahat[2] = ah16;
  ch.dsqrt_inv[0] = dsi64; ch.dsqrt_inv[1] = ds32; ch.dsqrt_inv[2] = ds16;
  oracle_cheb_apply(n, rowptr, col, &ch, u, y, z, w, w + n, w + 2 * n, w + 3 * n);
  free(buf);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Preconditioner apply z = M^-1 y in precision uz (Alg. 3).
 * Jacobi: z_i = dinv_i * y_i with dinv_i = fl64(1/a_ii) rounded to uz; for
 * FP16 the product of two FP16 numbers is formed exactly in FP32 and
 * rounded once.                                                            */
static void apply_precond(int mtype, int64_t n, int uz, const double* dinv_u,
                          const double* y, double* z) {
  for (int64_t i = 0; i < n; ++i) {
    if (mtype == OR_M_NONE) z[i] = y[i];
    else if (uz == OR_FP64) z[i] = dinv_u[i] * y[i];
    else z[i] = oracle_round(uz, mul32(dinv_u[i], y[i]));
  }
}

/* ------------------------------------------------------------------------ */
/* Alg. 3 scaling (R6): y_i = round_uz( fl_ur(omega * r_i) ).  With binary16
 * storage, counts[0] += the y_i with r_i != 0 that fall below binary16's
 * normal range (2^-14: subnormal or flushed to zero), counts[1] += the y_i
 * with r_i != 0 (diagnostics for the choice of omega; no effect on y).     */
static void scale_to_y(int64_t n, int uz, int ur, double omega, const double* r, double* y,
                       int64_t* counts) {
  double omega_r = oracle_round(ur, omega);
  for (int64_t i = 0; i < n; ++i) {
    double prod = (ur == OR_FP64) ? omega * r[i] : mul32(omega_r, r[i]);
    if (ur == OR_FP16) prod = oracle_round16(prod);
    y[i] = oracle_round(uz, prod);
    if (counts && uz == OR_FP16 && r[i] != 0.0) {
      counts[1]++;
      if (fabs(y[i]) < 6.103515625e-05) counts[0]++;   /* 2^-14 */
    }
  }
}

/* Alg. 3 scaling and preconditioning on their own, with M = none or Jacobi built from A as in
 * oracle_ampcg: z = M^-1 round_uz(omega r).  r must hold values of precision
 * ur.  Used by tests to check the device's preconditioner kernel.           */
int oracle_scale_precond(int64_t n, const int32_t* rowptr, const int32_t* col,
                         const double* val, int mtype, int uz, int ur, double omega,
                         const double* r, double* z) {
  double* w = (double*)malloc(sizeof(double) * (size_t)n * 2);
  if (!w) return OR_ERR_INVALID;
  double *dinv = w, *y = w + n;
  csr_diag(n, rowptr, col, val, dinv);
  for (int64_t i = 0; i < n; ++i) dinv[i] = oracle_round(uz, 1.0 / dinv[i]);
  scale_to_y(n, uz, ur, omega, r, y, NULL);
  apply_precond(mtype, n, uz, dinv, y, z);
  free(w);
  return OR_OK;
}

/* Same with the Chebyshev preconditioner (reading R8) built from A as in
 * oracle_ampcg: z = D^-1/2 P(Ahat) D^-1/2 round_uz(omega r).              */
int oracle_scale_cheb(int64_t n, const int32_t* rowptr, const int32_t* col,
                      const double* val, int degree, double lmin, double lmax, int uz,
                      int ur, double omega, const double* r, double* z) {
  int64_t nnz = rowptr[n];
  double* w = (double*)malloc(sizeof(double) * (size_t)(n * 7 + nnz));
  if (!w) return OR_ERR_INVALID;
  double *dg = w, *dsi = w + n, *y = w + 2 * n, *ah = w + 7 * n;
  csr_diag(n, rowptr, col, val, dg);
  for (int64_t i = 0; i < n; ++i) dsi[i] = 1.0 / sqrt(dg[i]);
  for (int64_t i = 0; i < n; ++i)
    for (int32_t kk = rowptr[i]; kk < rowptr[i + 1]; ++kk)
      ah[kk] = dsi[i] * val[kk] * dsi[col[kk]];
  scale_to_y(n, uz, ur, omega, r, y, NULL);
  int st = oracle_cheb_apply_public(n, nnz, rowptr, col, ah, dsi, degree, lmin, lmax, uz, y, z);
  free(w);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Alg. 3 search direction p_k = z_k + beta_{k-1} p_{k-1} in u_z (R7).  p holds
 * p_{k-1} in the precision of the previous iteration; it is first rounded to
 * u_z (a u_z change).  FP64: one FP64 fma.  FP32/FP16: one binary32 fma with
 * beta rounded to binary32, the result rounded once to u_z.  first: p_0 = z_0. */
void oracle_direction(int64_t n, int uz, int first, double beta, const double* z, double* p) {
  for (int64_t i = 0; i < n; ++i) {
    if (first) { p[i] = z[i]; continue; }
    double pold = oracle_round(uz, p[i]);
    if (uz == OR_FP64) p[i] = fma(beta, pold, z[i]);
    else p[i] = oracle_round(uz, fma32(oracle_round32(beta), pold, z[i]));
  }
}

/* Alg. 3 updates x_{k+1} = x_k + alpha p_k (FP64 fma; x is FP64) and
 * r_{k+1} = r_k - alpha q_k in u_r: FP64 fma, or one binary32 fma with alpha
 * rounded to binary32 and the result rounded to u_r (R7).                   */
void oracle_update_xr(int64_t n, int ur, double alpha, const double* p, const double* q,
                      double* x, double* r) {
  for (int64_t i = 0; i < n; ++i) x[i] = fma(alpha, p[i], x[i]);
  double alpha_r = oracle_round(ur == OR_FP64 ? OR_FP64 : OR_FP32, alpha);
  for (int64_t i = 0; i < n; ++i) {
    if (ur == OR_FP64) r[i] = fma(-alpha, q[i], r[i]);
    else r[i] = oracle_round(ur, fma32(-alpha_r, q[i], r[i]));
  }
}

/* ------------------------------------------------------------------------ */
/* PCG, Algorithm 1, native FP64, Jacobi or identity M.  Stops on the updated
 * residual ||r_{k+1}|| <= tol ||b||.  Returns iterations in res->iters.     */
int oracle_pcg64(int64_t n, const int32_t* rowptr, const int32_t* col,
                 const double* val, int mtype, const double* b, double* x,
                 double tol, int maxit, double* relres_hist, oracle_result* res) {
  double* r = (double*)malloc(sizeof(double) * (size_t)n * 5);
  if (!r) return OR_ERR_INVALID;
  double *z = r + n, *p = r + 2 * n, *q = r + 3 * n, *dinv = r + 4 * n;
  csr_diag(n, rowptr, col, val, dinv);
  for (int64_t i = 0; i < n; ++i) dinv[i] = 1.0 / dinv[i];
  memset(res, 0, sizeof(*res));
  res->switch_iter[0] = res->switch_iter[1] = res->switch_iter[2] = -1;
  oracle_residual64(n, rowptr, col, val, b, x, r);
  double nb = oracle_nrm2(n, b);
  double rn = oracle_nrm2(n, r);
  if (relres_hist) relres_hist[0] = rn / nb;
  double rho_prev = 0.0, beta = 0.0;
  int k = 0, status = OR_NOT_CONVERGED;
  if (rn <= tol * nb) status = OR_OK;
  for (k = 0; k < maxit && status == OR_NOT_CONVERGED; ++k) {
    for (int64_t i = 0; i < n; ++i) z[i] = (mtype == OR_M_NONE) ? r[i] : dinv[i] * r[i];
    double rho = oracle_dot(n, r, z);
    if (k > 0) beta = rho / rho_prev;
    for (int64_t i = 0; i < n; ++i) p[i] = (k == 0) ? z[i] : fma(beta, p[i], z[i]);
    for (int64_t i = 0; i < n; ++i) {
      double t = 0.0;
      for (int32_t kk = rowptr[i]; kk < rowptr[i + 1]; ++kk) t = fma(val[kk], p[col[kk]], t);
      q[i] = t;
    }
    double gamma = oracle_dot(n, q, p);
    if (!isfinite(rho) || !isfinite(gamma)) { status = OR_ERR_NONFINITE; break; }
    if (!(rho > 0.0) || !(gamma > 0.0)) { status = OR_ERR_BREAKDOWN; break; }
    double alpha = rho / gamma;
    for (int64_t i = 0; i < n; ++i) x[i] = fma(alpha, p[i], x[i]);
    for (int64_t i = 0; i < n; ++i) r[i] = fma(-alpha, q[i], r[i]);
    rn = oracle_nrm2(n, r);
    if (relres_hist) relres_hist[k + 1] = rn / nb;
    rho_prev = rho;
    if (rn <= tol * nb) status = OR_OK;
  }
  res->iters = k;
  res->status = status;
  res->converged = (status == OR_OK);
  res->updated_relres = rn / nb;
  oracle_residual64(n, rowptr, col, val, b, x, r);
  res->true_relres = oracle_nrm2(n, r) / nb;
  free(r);
  return status;
}

/* ------------------------------------------------------------------------ */
/* AMP-PCG, Algorithm 3 (DS-PCG, Algorithm 2, is the FIXED criterion with a
 * scale mode).  Every vector value is held in a double but only ever takes
 * values representable in the precision the algorithm assigns to it.
 *   mtype: OR_M_NONE / OR_M_JACOBI / OR_M_CHEBYSHEV (cheb_* then apply).
 *   relres_hist: length >= maxit + 1 (may be NULL); prec_hist: length >=
 *   maxit, byte (u_z << 4) | u_r per iteration (may be NULL).             */
int oracle_ampcg(int64_t n, const int32_t* rowptr, const int32_t* col,
                 const double* val, int mtype, int cheb_degree, double cheb_lmin,
                 double cheb_lmax, const double* b, double* x, double tol,
                 int maxit, const oracle_policy* pol, double* relres_hist,
                 uint8_t* prec_hist, oracle_result* res) {
  int64_t nnz = rowptr[n];
  memset(res, 0, sizeof(*res));
  res->switch_iter[0] = res->switch_iter[1] = res->switch_iter[2] = -1;
  if (n <= 0 || maxit < 0 || !(tol > 0.0)) { res->status = OR_ERR_INVALID; return OR_ERR_INVALID; }

  /* Matrix copies in each precision, Jacobi diagonal, Chebyshev data. */
  double* A[3];
  A[0] = (double*)val;
  A[1] = (double*)malloc(sizeof(double) * (size_t)nnz);
  A[2] = (double*)malloc(sizeof(double) * (size_t)nnz);
  double* dinv[3];
  double* vec = (double*)malloc(sizeof(double) * (size_t)n * 16);
  double* delta = (double*)malloc(sizeof(double) * (size_t)(maxit + 2));
  double *ahat[3] = {0, 0, 0}, *dsi[3] = {0, 0, 0};
  if (!A[1] || !A[2] || !vec || !delta) { res->status = OR_ERR_INVALID; return OR_ERR_INVALID; }
  for (int64_t k = 0; k < nnz; ++k) { A[1][k] = oracle_round32(val[k]); A[2][k] = oracle_round16(val[k]); }
  dinv[0] = vec; dinv[1] = vec + n; dinv[2] = vec + 2 * n;
  double *r = vec + 3 * n, *y = vec + 4 * n, *z = vec + 5 * n, *p = vec + 6 * n;
  double *q = vec + 7 * n, *t = vec + 8 * n, *w0 = vec + 9 * n;
  double *w1 = vec + 10 * n, *w2 = vec + 11 * n, *w3 = vec + 12 * n, *pw = vec + 13 * n;
  csr_diag(n, rowptr, col, val, dinv[0]);
  oracle_cheb ch;
  if (mtype == OR_M_CHEBYSHEV) {
    for (int u = 0; u < 3; ++u) {
      ahat[u] = (double*)malloc(sizeof(double) * (size_t)nnz);
      dsi[u] = (double*)malloc(sizeof(double) * (size_t)n);
    }
    for (int64_t i = 0; i < n; ++i) dsi[0][i] = 1.0 / sqrt(dinv[0][i]);
    for (int64_t i = 0; i < n; ++i)
      for (int32_t kk = rowptr[i]; kk < rowptr[i + 1]; ++kk)
        ahat[0][kk] = dsi[0][i] * val[kk] * dsi[0][col[kk]];
    for (int64_t kk = 0; kk < nnz; ++kk) { ahat[1][kk] = oracle_round32(ahat[0][kk]); ahat[2][kk] = oracle_round16(ahat[0][kk]); }
    for (int64_t i = 0; i < n; ++i) { dsi[1][i] = oracle_round32(dsi[0][i]); dsi[2][i] = oracle_round16(dsi[0][i]); }
    ch.degree = cheb_degree; ch.lmin = cheb_lmin; ch.lmax = cheb_lmax;
    for (int u = 0; u < 3; ++u) { ch.ahat[u] = ahat[u]; ch.dsqrt_inv[u] = dsi[u]; }
  }
  for (int64_t i = 0; i < n; ++i) dinv[0][i] = 1.0 / dinv[0][i];
  for (int64_t i = 0; i < n; ++i) { dinv[1][i] = oracle_round32(dinv[0][i]); dinv[2][i] = oracle_round16(dinv[0][i]); }

  /* Alg. 3 initialisation: r_0 = b - A x_0 (FP64), delta_0 = ||r_0||. */
  oracle_residual64(n, rowptr, col, val, b, x, r);
  double nb = oracle_nrm2(n, b);
  double tol_nb = tol * nb;
  delta[0] = oracle_nrm2(n, r);
  double maxr = oracle_maxabs(n, r);
  double maxr_prev = maxr;   /* max|r_{k-1}| (R20); r_0 for k = 0 */
  if (relres_hist) relres_hist[0] = delta[0] / nb;
  int status = OR_NOT_CONVERGED;
  if (!isfinite(nb) || !isfinite(delta[0])) status = OR_ERR_NONFINITE;
  else if (delta[0] <= tol_nb) status = OR_OK;

  int uz_prev = (pol->criterion == OR_CRIT_FIXED) ? pol->fixed_uz : pol->u0;
  int ur_prev = OR_FP64;     /* r_0 is FP64 */
  int uz_hist_prev = uz_prev, ur_hist_prev = OR_FP64;
  int p_prec = OR_FP64;
  double rho_prev = 0.0;
  int k = 0, refreshes = 0;
  int first = 1;             /* no search direction yet */
  for (k = 0; k < maxit && status == OR_NOT_CONVERGED; ++k) {
    /* indicator and precision selection */
    int uz, ur;
    if (pol->criterion == OR_CRIT_FIXED) {
      uz = pol->fixed_uz; ur = pol->fixed_ur;
    } else {
      double eta = (pol->criterion == OR_CRIT_WINDOW)
                       ? oracle_eta_window(delta, k, pol->d, pol->C)
                       : oracle_eta_linear(delta, k, pol->ell, pol->C);
      oracle_select(delta[k] / nb, pol->u0, pol->tau_zs, pol->tau_zh, eta, tol_nb, &uz, &ur);
      if (pol->latch) {
        if (uz < uz_prev) uz = uz_prev;
        if (ur < ur_prev) ur = ur_prev;
      }
    }
    if (uz != uz_hist_prev && uz == OR_FP32 && res->switch_iter[0] < 0) res->switch_iter[0] = k;
    if (uz != uz_hist_prev && uz == OR_FP16 && res->switch_iter[1] < 0) res->switch_iter[1] = k;
    if (ur != ur_hist_prev && ur == OR_FP32 && res->switch_iter[2] < 0) res->switch_iter[2] = k;
    uz_hist_prev = uz; ur_hist_prev = ur;
    if (prec_hist) prec_hist[k] = (uint8_t)((uz << 4) | ur);
    /* R10: r_k changes storage precision once, before y_k is formed. */
    if (ur != ur_prev)
      for (int64_t i = 0; i < n; ++i) r[i] = oracle_round(ur, r[i]);

    /* scaling: y_k = omega_k r_k, computed in u_r, stored in u_z (R5, R6,
       R20: the lagged mode takes max|r_{k-1}|, and max|r_k| on a retry) */
    int lag = pol->scale == OR_SCALE_LINF_POW2_LAG;
    double omega = oracle_scale(pol->scale, delta[k], lag ? maxr_prev : maxr);
    double rho = 0.0;
    for (int attempt = 0; attempt < 2; ++attempt) {
      int64_t counts[2] = {0, 0};
      scale_to_y(n, uz, ur, omega, r, y, counts);
      res->y16_small += counts[0];
      res->y16_total += counts[1];
      /* preconditioning: z_k = M^-1 y_k in u_z */
      if (mtype == OR_M_CHEBYSHEV)
        oracle_cheb_apply(n, rowptr, col, &ch, uz, y, z, w0, w1, w2, w3);
      else
        apply_precond(mtype, n, uz, dinv[uz], y, z);
      /* rho_k = r_k^T z_k (FP64) */
      rho = oracle_dot(n, r, z);
      if (isfinite(rho) || !lag || attempt == 1) break;
      omega = oracle_scale(OR_SCALE_LINF_POW2, delta[k], maxr);
      res->scale_retries++;
    }
    if (!isfinite(rho)) { status = OR_ERR_NONFINITE; break; }
    if (!(rho > 0.0)) { status = OR_ERR_BREAKDOWN; break; }
    /* beta_{k-1} = rho_k/rho_{k-1}; p_k = z_k + beta p_{k-1} in u_z;
       p_{k-1} is first brought to u_z when u_z changed.                   */
    double beta = first ? 0.0 : rho / rho_prev;
    oracle_direction(n, uz, first, beta, z, p);
    p_prec = uz;
    first = 0;
    /* q_k = A p_k in u_r (R7); gamma_k = q_k^T p_k (FP64) */
    oracle_spmv(n, rowptr, col, A[ur], ur, p, q);
    double gamma = oracle_dot(n, q, p);
    if (!isfinite(gamma)) { status = OR_ERR_NONFINITE; break; }
    if (!(gamma > 0.0)) { status = OR_ERR_BREAKDOWN; break; }
    /* alpha_k, x_{k+1}, r_{k+1} */
    double alpha = rho / gamma;
    oracle_update_xr(n, ur, alpha, p, q, x, r);
    ur_prev = ur; uz_prev = uz;
    rho_prev = rho;
    /* delta_{k+1} = ||r_{k+1}|| (FP64); max|r| for the next scale */
    delta[k + 1] = oracle_nrm2(n, r);
    maxr_prev = maxr;
    maxr = oracle_maxabs(n, r);
    if (relres_hist) relres_hist[k + 1] = delta[k + 1] / nb;
    if (!isfinite(delta[k + 1])) { status = OR_ERR_NONFINITE; k++; break; }
    /* stop on the updated residual */
    if (delta[k + 1] <= tol_nb) {
      status = OR_OK;
      if (refreshes < pol->verify_refresh && k + 1 < maxit) {
        /* R9: verify in FP64; if the true residual misses tol, replace r. */
        oracle_residual64(n, rowptr, col, val, b, x, t);
        double tr = oracle_nrm2(n, t);
        if (tr > tol_nb) {
          for (int64_t i = 0; i < n; ++i) r[i] = oracle_round(ur, t[i]);
          delta[k + 1] = oracle_nrm2(n, r);
          maxr = oracle_maxabs(n, r);
          if (relres_hist) relres_hist[k + 1] = delta[k + 1] / nb;
          refreshes++;
          status = (delta[k + 1] <= tol_nb) ? OR_OK : OR_NOT_CONVERGED;
        }
      }
    }
  }
  (void)p_prec; (void)pw;
  res->iters = k;
  res->status = status;
  res->converged = (status == OR_OK);
  res->refreshes = refreshes;
  res->updated_relres = delta[k] / nb;
  oracle_residual64(n, rowptr, col, val, b, x, t);
  res->true_relres = oracle_nrm2(n, t) / nb;
  free(A[1]); free(A[2]); free(vec); free(delta);
  for (int u = 0; u < 3; ++u) { free(ahat[u]); free(dsi[u]); }
  return status;
}

/* ------------------------------------------------------------------------ */
/* Replays the selector over a given sequence delta[0..m] exactly as the
 * solver does at each iteration k = 0..m (eta from the prefix, latch),
 * writing (u_z << 4) | u_r per k.  Pure scalar logic, for tests.           */
void oracle_selector_trace(const double* delta, int m, double nb, double tol,
                           const oracle_policy* pol, uint8_t* out) {
  int uz_prev = (pol->criterion == OR_CRIT_FIXED) ? pol->fixed_uz : pol->u0;
  int ur_prev = OR_FP64;
  double tol_nb = tol * nb;
  for (int k = 0; k <= m; ++k) {
    int uz, ur;
    if (pol->criterion == OR_CRIT_FIXED) { uz = pol->fixed_uz; ur = pol->fixed_ur; }
    else {
      double eta = (pol->criterion == OR_CRIT_WINDOW)
                       ? oracle_eta_window(delta, k, pol->d, pol->C)
                       : oracle_eta_linear(delta, k, pol->ell, pol->C);
      oracle_select(delta[k] / nb, pol->u0, pol->tau_zs, pol->tau_zh, eta, tol_nb, &uz, &ur);
      if (pol->latch) {
        if (uz < uz_prev) uz = uz_prev;
        if (ur < ur_prev) ur = ur_prev;
      }
    }
    out[k] = (uint8_t)((uz << 4) | ur);
    uz_prev = uz; ur_prev = ur;
  }
}

/* ------------------------------------------------------------------------ */
/* Adjoint gradient for the log-coefficient field (coefficient-field
 * workloads): with A x = b solved and A lambda = dL/dx, dL/da_ij = -lambda_i x_j;
 * pushing it through a_ij = -exp((th_i+th_j)/2) (i != j) and
 * a_ii = sum_{j != i} exp((th_i+th_j)/2) + nb_i exp(th_i) gives, per node,
 *   dL/dth_i = sum_{j != i} dL/dk_ij * k_ij/2 + dL/da_ii * nb_i exp(th_i),
 *   dL/dk_ij = dL/da_ii + dL/da_jj - dL/da_ij - dL/da_ji
 *            = -(lambda_i - lambda_j)(x_i - x_j),
 * with k_ij = -a_ij and nb_i exp(th_i) = sum_j a_ij.  Plain loops.          */
void oracle_grad_log_coeff(int64_t n, const int32_t* rowptr, const int32_t* col,
                           const double* val, const double* x, const double* lam,
                           double* out) {
  for (int64_t i = 0; i < n; ++i) {
    double g = 0.0, rowsum = 0.0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      int32_t j = col[k];
      rowsum = rowsum + val[k];
      if (j == i) continue;
      double dk = -((lam[i] - lam[j]) * (x[i] - x[j]));
      g = g + dk * (-val[k]) * 0.5;
    }
    out[i] = g + (-(lam[i] * x[i])) * rowsum;
  }
}
