// ampcg.cu -- host side of the C ABI declared in include/ampcg.h.
//
// A context owns the matrix in the sliced layout with its FP64/FP32 value
// copies, the Jacobi inverse diagonal in three precisions, every vector buffer
// of the iteration and one device state block.  A solve is: copy b and x_0 in,
// one initial-residual launch, then a CUDA graph of conditional nodes that
// repeats chunks of `graph_chunk` iterations (one persistent-kernel launch, or
// the pair's kernel sequence per iteration)
// of the current precision pair until the device sets `done`; then an FP64
// true-residual launch and one read of the state block.  The host synchronises once per solve (plus once per optional
// residual replacement).
#include <cuda.h>   // driver types only (context identity); no driver library is linked
#include <cuda_runtime.h>

#include <chrono>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <thread>
#include <string>
#include <vector>

#include "../../include/ampcg.h"
#include "batched.cuh"
#include "bsr.cuh"
#include "kernel_table.h"

using namespace ampcg;

namespace ampcg {
const void* loop_kernel(int uz, int ur, int mt, int it, bool fused) {
  if (mt == M_JACOBI) return fused ? loop_kernel_jacobi_fused(uz, ur, it) : loop_kernel_jacobi_plain(uz, ur, it);
  return fused ? loop_kernel_none_fused(uz, ur, it) : loop_kernel_none_plain(uz, ur, it);
}
const void* batched_kernel(int it, int bs) {
  if (bs == kBatchBlockSmall) return it ? batched_kernel_idx16_b512() : batched_kernel_idx32_b512();
  return it ? batched_kernel_idx16_b1024() : batched_kernel_idx32_b1024();
}
}  // namespace ampcg

namespace {

thread_local std::string g_err;

ampcg_status fail(ampcg_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CUDA_TRY(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      ampcg_status s_ = (e_ == cudaErrorMemoryAllocation) ? AMPCG_ERR_OOM : AMPCG_ERR_CUDA; \
      return fail(s_, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    }                                                                                   \
  } while (0)

constexpr int kBlock = 256;
constexpr int kLoopChunk = 256;   // default iterations per persistent-kernel launch
constexpr int kSeqChunk = 16;     // default iterations per repeat of the kernel sequence

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
ampcg_status dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  CUDA_TRY(cudaMalloc((void**)p, count * sizeof(T)));
  return AMPCG_OK;
}

}  // namespace

// One kernel launch of an iteration: function, launch shape, argument list
// kind, timing slot (0 precondition, 1 search direction, 2 SpMV, 3 update)
// and, for a Chebyshev step, its index and constants.
enum { KA_ELEM = 0, KA_SPMV, KA_UPD, KA_CINIT, KA_CSTEP, KA_CFINAL, KA_LOOP, KA_BSPMV, KA_BCSTEP };
struct Launch {
  const void* fn;
  int grid, smem, kind, slot, j;
  double c1, c2;
  bool coop;   // cooperative launch (the kernel has a grid barrier)
  int block = kBlock;
};

struct ampcg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t cap_stream = nullptr;
  int64_t n = 0, nnz = 0, nslices = 0;
  int idx16 = 0;  // 1: int16 column offsets
  int maxw = 0;   // largest slice width
  int mtype = M_JACOBI;
  // matrix
  int* rowptr = nullptr;  // CSR row pointer (maps sliced entries to CSR order)
  long long* off = nullptr;
  int* width = nullptr;
  int* cabs = nullptr;
  short* coff = nullptr;
  double* v64 = nullptr;
  float* v32 = nullptr;
  double* dinv64 = nullptr;
  float* dinv32 = nullptr;
  __half* dinv16 = nullptr;
  // vectors
  double *x = nullptr, *b = nullptr, *r64 = nullptr, *t = nullptr;
  float* r32 = nullptr;
  void *z = nullptr, *p0 = nullptr, *p1 = nullptr, *q = nullptr;
  double* part = nullptr;
  unsigned long long* pmax = nullptr;
  GridSumBarrier* bar = nullptr;  // barriers of the cooperative launches (k_precond_dir, k_loop; one per pair), zeroed per solve
  DevState* st = nullptr;       // device
  DevState* hst = nullptr;      // pinned host mirror
  double* dhist = nullptr;      // delta history
  unsigned char* phist = nullptr;
  int hist_cap = 0;
  // launch shapes
  int g_elem = 1, g_rows = 1, g_max = 1;
  // iteration kernels per phase (2 u_z + u_r), in launch order
  std::vector<Launch> seq[6];
  // k_loop per precision pair (Jacobi or none, slices at most kStageW wide):
  // the device loop and the timed path launch it instead of seq
  int stream_hint = 0;    // Sell::stream_hint
  int64_t stored = 0;     // stored entries of the sliced layout
  short* pat = nullptr;   // Sell::pat
  unsigned char* rmask = nullptr;  // Sell::rmask
  Launch loop[2][6];      // [fused][pair]: four or three grid barriers per iteration
  bool loop_ok = true;    // every pair's k_loop configured (set while building)
  bool use_loop = false;
  // k_loop form per pair for the scale modes that allow the three-barrier
  // one ([0] SCALE_NONE, [1] LINF_POW2_LAG): -1 automatic (three barriers),
  // 0 four, 1 three; set by ampcg_tune / ampcg_set_tuning
  // per scale slot (NONE, lagged power of two, exact power of two; see scale_slot)
  int loop_form[3][6] = {{-1, -1, -1, -1, -1, -1}, {-1, -1, -1, -1, -1, -1}, {-1, -1, -1, -1, -1, -1}};
  unsigned fused_mask = 0;   // the current solve's forms: bit ph set = three-barrier k_loop for pair ph
  int batch_block = 0;       // block size of the batched kernel for batches led by this context (0: 1024)
  // Chebyshev preconditioner data (reading R8)
  int cheb_m = 0;
  int cheb_auto = 0;            // interval from the Gershgorin bound
  double cheb_lmin = 0.0, cheb_lmax = 0.0, cheb_inv_theta = 0.0;
  std::vector<double> cheb_c1, cheb_c2;  // per step j = 1..m-1
  double* ah64 = nullptr;
  float* ah32 = nullptr;
  __half* ah16 = nullptr;
  unsigned* ahp = nullptr;      // packed FP16 value + int16 offset (int16-offset matrices)
  double* ds64 = nullptr;
  float* ds32 = nullptr;
  __half* ds16 = nullptr;
  void *cres = nullptr, *cd0 = nullptr, *cd1 = nullptr, *cu = nullptr;
  Cheb cheb() const {
    Cheb C;
    C.ah64 = ah64; C.ah32 = ah32; C.ah16 = ah16; C.ahp = ahp;
    C.ds64 = ds64; C.ds32 = ds32; C.ds16 = ds16;
    C.res = cres; C.d[0] = cd0; C.d[1] = cd1; C.u = cu;
    C.inv_theta = cheb_inv_theta;
    return C;
  }
  // block-row layout of a 3 x 3 block matrix (bsr.cuh), when created from
  // block CSR with bs = 3 and wide rows
  bool bs3 = false;
  int64_t nb3 = 0, nbs3 = 0, bstored = 0;
  long long* boff = nullptr;
  int* bw = nullptr;
  int* bcol3 = nullptr;
  double* bv64 = nullptr;
  float* bv32 = nullptr;
  double* bah64 = nullptr;
  float* bah32 = nullptr;
  __half* bah16 = nullptr;
  BSell bsell() const {
    BSell A;
    A.nb = nb3;
    A.nbs = nbs3;
    A.boff = boff;
    A.bw = bw;
    A.bcol = bcol3;
    A.v64 = bv64;
    A.v32 = bv32;
    A.ah64 = bah64;
    A.ah32 = bah32;
    A.ah16 = bah16;
    return A;
  }
  // device-side loop graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int graph_chunk = 0;
  unsigned graph_fused = 0;

  Sell sell() const {
    Sell A;
    A.n = n;
    A.nslices = nslices;
    A.maxw = maxw;
    A.off = off;
    A.width = width;
    A.cabs = idx16 ? nullptr : cabs;
    A.coff = idx16 ? coff : nullptr;
    A.v64 = v64;
    A.v32 = v32;
    A.stream_hint = stream_hint;
    A.pat = idx16 ? pat : nullptr;
    A.rmask = idx16 ? rmask : nullptr;
    return A;
  }
  Bufs bufs() const {
    Bufs B;
    B.x = x;
    B.b = b;
    B.r64 = r64;
    B.r32 = r32;
    B.z = z;
    B.p[0] = p0;
    B.p[1] = p1;
    B.q = q;
    B.t = t;
    B.dinv64 = dinv64;
    B.dinv32 = dinv32;
    B.dinv16 = dinv16;
    B.part = part;
    B.pmax = pmax;
    B.bar = bar;
    return B;
  }
};

static void release(ampcg_ctx* c) {
  if (!c) return;
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  void* ptrs[] = {c->ah64, c->ah32, c->ah16, c->ahp, c->ds64, c->ds32, c->ds16, c->cres, c->cd0, c->cd1, c->cu,
                  c->rowptr, c->off, c->width, c->cabs, c->coff, c->pat, c->rmask, c->v64, c->v32, c->dinv64, c->dinv32,
                  c->dinv16, c->x, c->b, c->r64, c->t, c->r32, c->z, c->p0, c->p1, c->q,
                  c->part, c->pmax, c->bar, c->st, c->dhist, c->phist, c->boff, c->bw, c->bcol3, c->bv64,
                  c->bv32, c->bah64, c->bah32, c->bah16};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->hst) cudaFreeHost(c->hst);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

static int occ_grid(const void* kern, int sms, int64_t work_threads, int smem = 0, int block = kBlock) {
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 4;
  }
  if (per_sm < 1) per_sm = 1;
  int64_t g = (int64_t)sms * per_sm;
  int64_t need = (work_threads + block - 1) / block;
  if (need < 1) need = 1;
  return (int)(g < need ? g : need);
}

extern "C" {

void ampcg_policy_default(ampcg_policy* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->u0 = AMPCG_FP16;
  p->criterion = AMPCG_CRIT_LINEAR;
  p->d = 10;
  p->ell = 5;
  p->C = 1.0;
  p->tau_zs = 1e-4;
  p->tau_zh = 1e-6;
  p->scale = AMPCG_SCALE_LINF_POW2;
  p->latch = 1;
  p->verify_refresh = 0;
  p->fixed_uz = AMPCG_FP64;
  p->fixed_ur = AMPCG_FP64;
  p->graph_chunk = 0;   // automatic: kLoopChunk or kSeqChunk
}

const char* ampcg_status_string(int s) {
  switch (s) {
    case AMPCG_OK: return "AMPCG_OK";
    case AMPCG_NOT_CONVERGED: return "AMPCG_NOT_CONVERGED";
    case AMPCG_ERR_INVALID_ARG: return "AMPCG_ERR_INVALID_ARG";
    case AMPCG_ERR_NOT_SPD: return "AMPCG_ERR_NOT_SPD";
    case AMPCG_ERR_BREAKDOWN: return "AMPCG_ERR_BREAKDOWN";
    case AMPCG_ERR_NONFINITE: return "AMPCG_ERR_NONFINITE";
    case AMPCG_ERR_CUDA: return "AMPCG_ERR_CUDA";
    case AMPCG_ERR_OOM: return "AMPCG_ERR_OOM";
    case AMPCG_ERR_TIMEOUT: return "AMPCG_ERR_TIMEOUT";
    case AMPCG_ERR_NO_DEVICE: return "AMPCG_ERR_NO_DEVICE";
    case AMPCG_ERR_UNSUPPORTED: return "AMPCG_ERR_UNSUPPORTED";
    default: return "AMPCG_UNKNOWN_STATUS";
  }
}

const char* ampcg_last_error(void) { return g_err.c_str(); }

int64_t ampcg_rows(ampcg_t c) { return c ? c->n : -1; }

ampcg_status ampcg_layout_stats(ampcg_t c, ampcg_layout* out) {
  if (!c || !out) return fail(AMPCG_ERR_INVALID_ARG, "NULL argument");
  memset(out, 0, sizeof(*out));
  out->n = c->n;
  out->nslices = c->nslices;
  out->stored = c->stored;
  out->maxw = c->maxw;
  out->idx16 = c->idx16;
  out->stream_hint = c->stream_hint;
  out->block3 = c->bs3 ? 1 : 0;
  if (c->pat) {
    std::vector<short> pat((size_t)c->nslices * kStageW);
    std::vector<int> w((size_t)c->nslices);
    CUDA_TRY(cudaMemcpyAsync(pat.data(), c->pat, pat.size() * sizeof(short), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaMemcpyAsync(w.data(), c->width, w.size() * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (int64_t s = 0; s < c->nslices; ++s)
      if (pat[(size_t)s * kStageW] != kNoPat) out->stored_uniform += 32ll * w[(size_t)s];
  }
  return AMPCG_OK;
}

void ampcg_destroy(ampcg_t c) {
  if (!c) return;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  release(c);
  cudaSetDevice(dev);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// create

static ampcg_status build_sequences(ampcg_ctx* c, int sms);
static ampcg_status cheb_prepare(ampcg_ctx* c);

static ampcg_status create_impl(ampcg_ctx* c, int64_t n, int64_t nnz, const int32_t* rowptr,
                                const int32_t* colind, const double* vals) {
  cudaStream_t s = c->stream;
  // stage CSR on the device
  const int* d_rp = (const int*)rowptr;
  const int* d_ci = (const int*)colind;
  const double* d_v = vals;
  int* t_rp = nullptr;
  int* t_ci = nullptr;
  double* t_v = nullptr;
  int* rowlen = nullptr;
  double* diag = nullptr;
  int* flags = nullptr;
  long long* total = nullptr;
  ampcg_status st = AMPCG_OK;
  auto cleanup = [&]() {
    if (t_rp) cudaFree(t_rp);
    if (t_ci) cudaFree(t_ci);
    if (t_v) cudaFree(t_v);
    if (rowlen) cudaFree(rowlen);
    if (diag) cudaFree(diag);
    if (flags) cudaFree(flags);
    if (total) cudaFree(total);
  };
#define TRY(x)                  \
  do {                          \
    st = (x);                   \
    if (st != AMPCG_OK) {       \
      cleanup();                \
      return st;                \
    }                           \
  } while (0)
#define CTRY(call)                                                                              \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) {                                                                    \
      cleanup();                                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? AMPCG_ERR_OOM : AMPCG_ERR_CUDA,             \
                  "%s failed: %s", #call, cudaGetErrorString(e_));                              \
    }                                                                                           \
  } while (0)

  if (!is_device_ptr(rowptr)) {
    TRY(dalloc(&t_rp, n + 1));
    CTRY(cudaMemcpyAsync(t_rp, rowptr, (n + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
    d_rp = t_rp;
  }
  if (!is_device_ptr(colind)) {
    TRY(dalloc(&t_ci, nnz));
    if (nnz) CTRY(cudaMemcpyAsync(t_ci, colind, nnz * sizeof(int), cudaMemcpyHostToDevice, s));
    d_ci = t_ci;
  }
  if (!is_device_ptr(vals)) {
    TRY(dalloc(&t_v, nnz));
    if (nnz) CTRY(cudaMemcpyAsync(t_v, vals, nnz * sizeof(double), cudaMemcpyHostToDevice, s));
    d_v = t_v;
  }
  TRY(dalloc(&c->rowptr, n + 1));
  CTRY(cudaMemcpyAsync(c->rowptr, d_rp, (n + 1) * sizeof(int), cudaMemcpyDeviceToDevice, s));
  TRY(dalloc(&rowlen, n));
  TRY(dalloc(&diag, n));
  TRY(dalloc(&flags, 2));
  TRY(dalloc(&total, 2));
  CTRY(cudaMemsetAsync(flags, 0, 2 * sizeof(int), s));
  int gb = (int)((n + kBlock - 1) / kBlock);
  k_csr_scan_rows<<<gb, kBlock, 0, s>>>(n, nnz, d_rp, d_ci, d_v, rowlen, diag, flags, flags + 1);
  CTRY(cudaGetLastError());
  int hflags[2] = {0, 0};
  CTRY(cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, s));
  CTRY(cudaStreamSynchronize(s));
  if (hflags[0] & 3) {
    cleanup();
    return fail(AMPCG_ERR_INVALID_ARG, "CSR structure invalid (flags %d): rowptr must be "
                "nondecreasing from 0 to nnz, columns in [0,n) strictly increasing per row", hflags[0]);
  }
  if (hflags[0] & 8) {
    cleanup();
    return fail(AMPCG_ERR_NONFINITE, "matrix has non-finite values");
  }
  if (hflags[0] & 4) {
    cleanup();
    return fail(AMPCG_ERR_NOT_SPD, "a diagonal entry is missing or not positive: A is not SPD");
  }
  c->idx16 = (hflags[1] <= 32767) ? 1 : 0;
  c->nslices = (n + 31) / 32;
  TRY(dalloc(&c->width, c->nslices));
  TRY(dalloc(&c->off, c->nslices));
  int gs = (int)((c->nslices + kBlock - 1) / kBlock);
  k_slice_width<<<gs, kBlock, 0, s>>>(n, c->nslices, rowlen, c->width);
  k_slice_offsets<<<1, 1024, 0, s>>>(c->nslices, c->width, c->off, total);
  CTRY(cudaGetLastError());
  long long tot2[2] = {0, 0};
  CTRY(cudaMemcpyAsync(tot2, total, sizeof(tot2), cudaMemcpyDeviceToHost, s));
  CTRY(cudaStreamSynchronize(s));
  long long stored = tot2[0];
  c->stored = stored;
  c->maxw = (int)tot2[1];
  {
    // the matrix (binary32 copy) and ~40 bytes per row of vectors would not
    // fit in L2 together: stream the matrix with an evict-first hint
    const double mbytes = (double)stored * (4 + (c->idx16 ? 2 : 4)) + 40.0 * (double)n;
    c->stream_hint = mbytes > 96.0 * (1 << 20) ? 1 : 0;
  }
  if (c->idx16) TRY(dalloc(&c->coff, stored));
  else TRY(dalloc(&c->cabs, stored));
  TRY(dalloc(&c->v64, stored));
  TRY(dalloc(&c->v32, stored));
  int64_t rows_pad = c->nslices * 32;
  if (c->idx16) {
    TRY(dalloc(&c->pat, (size_t)c->nslices * kStageW));
    TRY(dalloc(&c->rmask, (size_t)rows_pad));
    k_slice_pattern<<<gs, kBlock, 0, s>>>(n, c->nslices, d_rp, d_ci, c->width, c->pat);
  }
  k_fill_sell<<<(int)((rows_pad + kBlock - 1) / kBlock), kBlock, 0, s>>>(
      n, d_rp, d_ci, d_v, c->off, c->width, c->pat, c->cabs, c->coff, c->v64, c->v32, c->rmask);
  int64_t npad = (n + 63) / 64 * 64;  // per-row arrays: whole 8-element vectors in bounds
  TRY(dalloc(&c->dinv64, npad));
  TRY(dalloc(&c->dinv32, npad));
  TRY(dalloc(&c->dinv16, npad));
  k_jacobi<<<gb, kBlock, 0, s>>>(n, diag, c->dinv64, c->dinv32, c->dinv16);
  CTRY(cudaGetLastError());
  // iteration buffers (padded like dinv)
  TRY(dalloc(&c->x, npad));
  TRY(dalloc(&c->b, npad));
  TRY(dalloc(&c->r64, npad));
  TRY(dalloc(&c->t, npad));
  TRY(dalloc(&c->r32, npad));
  double* tmp;
  TRY(dalloc(&tmp, npad)); c->z = tmp;
  TRY(dalloc(&tmp, npad)); c->p0 = tmp;
  TRY(dalloc(&tmp, npad)); c->p1 = tmp;
  TRY(dalloc(&tmp, npad)); c->q = tmp;
  CTRY(cudaMemsetAsync(c->p0, 0, npad * 8, s));
  CTRY(cudaMemsetAsync(c->p1, 0, npad * 8, s));
  // launch shapes
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  if (c->mtype == M_CHEBYSHEV) {
    TRY(dalloc(&c->ah64, stored));
    TRY(dalloc(&c->ah32, stored));
    TRY(dalloc(&c->ah16, stored));
    if (c->idx16) TRY(dalloc(&c->ahp, stored));
    TRY(dalloc(&c->ds64, npad));
    TRY(dalloc(&c->ds32, npad));
    TRY(dalloc(&c->ds16, npad));
    TRY(dalloc(&tmp, npad)); c->cres = tmp;
    TRY(dalloc(&tmp, npad)); c->cd0 = tmp;
    TRY(dalloc(&tmp, npad)); c->cd1 = tmp;
    TRY(dalloc(&tmp, npad)); c->cu = tmp;
    TRY(cheb_prepare(c));
  }
  TRY(build_sequences(c, sms));
  c->g_elem = occ_grid((const void*)k_refresh, sms, n);
  c->g_rows = occ_grid(c->idx16 ? (const void*)k_true_residual<1> : (const void*)k_true_residual<0>, sms,
                       rows_pad);
  c->g_max = c->g_elem > c->g_rows ? c->g_elem : c->g_rows;
  for (int ph = 0; ph < 6; ++ph) {
    for (const Launch& L : c->seq[ph])
      if (L.grid > c->g_max) c->g_max = L.grid;
    for (int f = 0; f < 2; ++f)
      if (c->use_loop && c->loop[f][ph].grid > c->g_max) c->g_max = c->loop[f][ph].grid;
  }
  int gi = occ_grid((const void*)k_init<0>, sms, rows_pad);
  if (gi > c->g_max) c->g_max = gi;
  TRY(dalloc(&c->part, (size_t)c->g_max * 6));   // the grid barriers' partials (device_util.cuh)
  TRY(dalloc(&c->pmax, (size_t)c->g_max * 2));   // two halves for the grid barriers
  TRY(dalloc(&c->bar, 12));
  TRY(dalloc(&c->st, 1));
  CTRY(cudaMallocHost((void**)&c->hst, sizeof(DevState)));
  memset(c->hst, 0, sizeof(DevState));
  CTRY(cudaMemsetAsync(c->st, 0, sizeof(DevState), s));
  CTRY(cudaStreamSynchronize(s));
  cleanup();
#undef TRY
#undef CTRY
  return AMPCG_OK;
}

extern "C" ampcg_status ampcg_create_csr(ampcg_t* out, int64_t n, int64_t nnz,
                                         const int32_t* rowptr, const int32_t* colind,
                                         const double* vals, const ampcg_precond_spec* M,
                                         void* cuda_stream) {
  if (!out) return fail(AMPCG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(AMPCG_ERR_NO_DEVICE, "no CUDA device visible");
  }
  if (n <= 0 || n > (int64_t)0x7fffffe0 || nnz < 0 || nnz > (int64_t)0x7fffffff)
    return fail(AMPCG_ERR_INVALID_ARG, "n must be in [1, 2^31-32) and nnz in [0, 2^31)");
  if (!rowptr || (nnz > 0 && (!colind || !vals)))
    return fail(AMPCG_ERR_INVALID_ARG, "NULL CSR array");
  int mtype = M ? M->type : AMPCG_M_JACOBI;
  if (mtype != AMPCG_M_NONE && mtype != AMPCG_M_JACOBI && mtype != AMPCG_M_CHEBYSHEV)
    return fail(AMPCG_ERR_INVALID_ARG, "unknown preconditioner type %d", mtype);
  if (mtype == AMPCG_M_CHEBYSHEV) {
    if (M->degree < 1 || M->degree > 64) return fail(AMPCG_ERR_INVALID_ARG, "Chebyshev degree must be in [1, 64]");
    if (M->lmax > 0.0 && !(M->lmin > 0.0 && M->lmin < M->lmax) && M->lmin != 0.0)
      return fail(AMPCG_ERR_INVALID_ARG, "Chebyshev interval needs 0 < lmin < lmax (or lmin = 0)");
  }
  ampcg_ctx* c = new ampcg_ctx();
  cudaGetDevice(&c->device);
  c->n = n;
  c->nnz = nnz;
  c->mtype = mtype;
  if (mtype == M_CHEBYSHEV) {
    c->cheb_m = M->degree;
    c->cheb_auto = !(M->lmax > 0.0);
    c->cheb_lmax = M->lmax;
    c->cheb_lmin = (M->lmin > 0.0) ? M->lmin : M->lmax / 30.0;
  }
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return fail(AMPCG_ERR_CUDA, "cudaStreamCreate failed");
    }
    c->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    release(c);
    return fail(AMPCG_ERR_CUDA, "cudaStreamCreate failed");
  }
  ampcg_status s = create_impl(c, n, nnz, rowptr, colind, vals);
  if (s != AMPCG_OK) {
    if (c->stream) cudaStreamSynchronize(c->stream);
    release(c);
    return s;
  }
  *out = c;
  return AMPCG_OK;
}

// ---------------------------------------------------------------------------
// solve

static ampcg_status ensure_hist(ampcg_ctx* c, int maxit) {
  int need = maxit + 2;
  if (need <= c->hist_cap) return AMPCG_OK;
  if (c->dhist) cudaFree(c->dhist);
  if (c->phist) cudaFree(c->phist);
  c->dhist = nullptr;
  c->phist = nullptr;
  c->hist_cap = 0;
  ampcg_status s;
  if ((s = dalloc(&c->dhist, need)) != AMPCG_OK) return s;
  if ((s = dalloc(&c->phist, need)) != AMPCG_OK) return s;
  c->hist_cap = need;
  return AMPCG_OK;
}

// Launch sequence of each phase (2 u_z + u_r): the precondition step (one
// kernel, or init + m-1 steps + final for Chebyshev), then search direction,
// SpMV, update.
template <int MT, int IT, int UZ, int UR>
static void phase_seq(ampcg_ctx* c, int sms, std::vector<Launch>& v) {
  const int64_t n = c->n, nvec = (n + 7) / 8;
  auto add = [&](const void* fn, int kind, int slot, int64_t work, int smem, int j = 0, double c1 = 0,
                 double c2 = 0) {
    Launch L;
    L.fn = fn; L.kind = kind; L.slot = slot; L.j = j; L.c1 = c1; L.c2 = c2; L.smem = smem; L.coop = false;
    if (smem > 0) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    L.grid = occ_grid(fn, sms, work, smem);
    v.push_back(L);
  };
  v.clear();
  if constexpr (MT == M_CHEBYSHEV) {
    add((const void*)k_cheb_init<UZ, UR>, KA_CINIT, 0, n, 0);
    for (int j = 1; j < c->cheb_m; ++j) {
      if (c->bs3)
        add(bsr_cheb_kernel(UZ, UR), KA_BCSTEP, 0, c->nbs3 * 32, 0, j, c->cheb_c1[j - 1], c->cheb_c2[j - 1]);
      else
        add((const void*)k_cheb_step<UZ, UR, IT>, KA_CSTEP, 0, c->nslices * 32, 0, j, c->cheb_c1[j - 1],
            c->cheb_c2[j - 1]);
    }
    add((const void*)k_cheb_final<UZ, UR>, KA_CFINAL, 0, n, 0);
    add((const void*)k_axpy<UZ, UR>, KA_ELEM, 1, nvec, 0);
  } else {
    // precondition, rho, beta and the search direction in one cooperative
    // launch (its grid is at most the resident blocks: occ_grid)
    add((const void*)k_precond_dir<UZ, UR, MT>, KA_ELEM, 0, nvec, 0);
    v.back().coop = true;
  }
  const bool wide = c->maxw > kStageW;
  const int sm = wide ? 0 : staged_smem_bytes<UR, IT>();
  if (c->bs3)
    add(bsr_spmv_kernel(UZ, UR), KA_BSPMV, 2, c->nbs3 * 32, 0);
  else
    add(wide ? (const void*)k_spmv<UZ, UR, IT, true> : (const void*)k_spmv<UZ, UR, IT, false>, KA_SPMV, 2,
        c->nslices * 32, sm);
  if (sm > 0) {
    // staged SpMV: a warp takes at most 32 slices, so at least nslices/32 warps
    int need = (int)((c->nslices + 32 * 8 - 1) / (32 * 8));
    if (v.back().grid < need) v.back().grid = need;
  }
  add((const void*)k_update<UZ, UR>, KA_UPD, 3, nvec, 0);
  if constexpr (MT != M_CHEBYSHEV) {
    if (!wide) {
      // the whole iteration loop in one cooperative launch, one block of
      // kLoopBlock threads per SM (a context whose pairs cannot all be
      // configured keeps the kernel sequences)
      for (int f = 0; f < 2; ++f) {
        const void* fn = loop_kernel(UZ, UR, MT, IT, f != 0);
        const int lsm = LoopStageCfg<UR, IT>::kBytes;
        int per_sm = 0;
        if (!fn || cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, lsm) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kLoopBlock, lsm) != cudaSuccess ||
            per_sm < 1) {
          cudaGetLastError();
          c->loop_ok = false;
        } else {
          Launch L;
          L.fn = fn; L.kind = KA_LOOP; L.slot = 0; L.j = 0; L.c1 = 0; L.c2 = 0; L.smem = lsm; L.coop = true;
          L.block = kLoopBlock;
          L.grid = occ_grid(fn, sms, c->nslices * 32, lsm, kLoopBlock);
          c->loop[f][2 * UZ + UR] = L;
        }
      }
    } else {
      c->loop_ok = false;
    }
  }
}

template <int MT, int IT>
static void build_sequences_t(ampcg_ctx* c, int sms) {
  c->loop_ok = MT != M_CHEBYSHEV;
  phase_seq<MT, IT, P64, P64>(c, sms, c->seq[0]);
  phase_seq<MT, IT, P64, P32>(c, sms, c->seq[1]);
  phase_seq<MT, IT, P32, P64>(c, sms, c->seq[2]);
  phase_seq<MT, IT, P32, P32>(c, sms, c->seq[3]);
  phase_seq<MT, IT, P16, P64>(c, sms, c->seq[4]);
  phase_seq<MT, IT, P16, P32>(c, sms, c->seq[5]);
  c->use_loop = c->loop_ok;
}

static ampcg_status build_sequences(ampcg_ctx* c, int sms) {
  if (c->mtype == M_NONE) { if (c->idx16) build_sequences_t<M_NONE, 1>(c, sms); else build_sequences_t<M_NONE, 0>(c, sms); }
  else if (c->mtype == M_JACOBI) { if (c->idx16) build_sequences_t<M_JACOBI, 1>(c, sms); else build_sequences_t<M_JACOBI, 0>(c, sms); }
  else { if (c->idx16) build_sequences_t<M_CHEBYSHEV, 1>(c, sms); else build_sequences_t<M_CHEBYSHEV, 0>(c, sms); }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(AMPCG_ERR_CUDA, "kernel attributes: %s", cudaGetErrorString(e));
  return AMPCG_OK;
}

// Ahat, D^-1/2 (three precisions each), the interval and the Chebyshev
// constants (reading R8; the same FP64 expressions as the oracle).  With an
// automatic interval, lmax is the Gershgorin bound max_i sum_j |ahat_ij| (an
// upper bound of the spectrum, so M stays SPD) and lmin = lmax / 30.
static ampcg_status cheb_prepare(ampcg_ctx* c) {
  cudaStream_t s = c->stream;
  unsigned long long* gk = nullptr;
  ampcg_status st = dalloc(&gk, 1);
  if (st != AMPCG_OK) return st;
  Sell A = c->sell();
  const int gs = (int)((c->nslices * 32 + kBlock - 1) / kBlock < 148 * 8 ? (c->nslices * 32 + kBlock - 1) / kBlock : 148 * 8);
  cudaError_t e = cudaMemsetAsync(gk, 0, sizeof(*gk), s);
  if (e == cudaSuccess) {
    if (c->idx16) {
      k_cheb_setup<1><<<gs, kBlock, 0, s>>>(A, c->ah64, c->ah32, c->ah16, c->ds64, c->ds32, c->ds16, gk);
      k_cheb_setup2<1><<<gs, kBlock, 0, s>>>(A, c->ds64, c->ah64, c->ah32, c->ah16, c->ahp, gk);
    } else {
      k_cheb_setup<0><<<gs, kBlock, 0, s>>>(A, c->ah64, c->ah32, c->ah16, c->ds64, c->ds32, c->ds16, gk);
      k_cheb_setup2<0><<<gs, kBlock, 0, s>>>(A, c->ds64, c->ah64, c->ah32, c->ah16, nullptr, gk);
    }
    e = cudaGetLastError();
  }
  unsigned long long hk = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hk, gk, sizeof(hk), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(gk);
  if (e != cudaSuccess) return fail(AMPCG_ERR_CUDA, "Chebyshev setup: %s", cudaGetErrorString(e));
  if (c->cheb_auto) {
    double g;
    memcpy(&g, &hk, sizeof(g));
    c->cheb_lmax = g;
    c->cheb_lmin = g / 30.0;
  }
  double a = c->cheb_lmin, bb = c->cheb_lmax;
  double theta = (bb + a) / 2.0, delt = (bb - a) / 2.0;
  double sigma = theta / delt;
  double rho = 1.0 / sigma;
  c->cheb_inv_theta = 1.0 / theta;
  c->cheb_c1.assign(c->cheb_m > 1 ? c->cheb_m - 1 : 0, 0.0);
  c->cheb_c2.assign(c->cheb_m > 1 ? c->cheb_m - 1 : 0, 0.0);
  for (int j = 1; j < c->cheb_m; ++j) {
    double rho_next = 1.0 / (2.0 * sigma - rho);
    c->cheb_c1[j - 1] = rho_next * rho;
    c->cheb_c2[j - 1] = 2.0 * rho_next / delt;
    rho = rho_next;
  }
  return AMPCG_OK;
}

// Argument storage for one launch (kernel parameters are copied at launch or
// graph-node creation, so one pack is reused).
struct ArgPack {
  Bufs B;
  Sell A;
  BSell BA;
  Cheb C;
  int64_t n;
  DevState* st;
  int j, iters;
  double c1, c2;
  void* a[8];
  explicit ArgPack(const ampcg_ctx* c, int it = 1)
      : B(c->bufs()), A(c->sell()), BA(c->bsell()), C(c->cheb()), n(c->n), st(c->st), j(0), iters(it), c1(0),
        c2(0) {}
  void** args(const Launch& L) {
    switch (L.kind) {
      case KA_ELEM:
      case KA_UPD: a[0] = &B; a[1] = &n; a[2] = &st; break;
      case KA_SPMV: a[0] = &A; a[1] = &B; a[2] = &st; break;
      case KA_LOOP: a[0] = &A; a[1] = &B; a[2] = &n; a[3] = &st; a[4] = &iters; break;
      case KA_CINIT:
      case KA_CFINAL: a[0] = &B; a[1] = &C; a[2] = &n; a[3] = &st; break;
      case KA_CSTEP:
        j = L.j; c1 = L.c1; c2 = L.c2;
        a[0] = &A; a[1] = &C; a[2] = &st; a[3] = &j; a[4] = &c1; a[5] = &c2;
        break;
      case KA_BSPMV: a[0] = &BA; a[1] = &B; a[2] = &st; break;
      case KA_BCSTEP:
        j = L.j; c1 = L.c1; c2 = L.c2;
        a[0] = &BA; a[1] = &C; a[2] = &st; a[3] = &j; a[4] = &c1; a[5] = &c2;
        break;
    }
    return a;
  }
};

// One iteration of phase ph launched kernel by kernel on stream s; with ev,
// ev[slot] is recorded before the first kernel of each slot and ev[4] after
// the last kernel.
// The launches of one iteration of phase ph: k_loop (one iteration) where it
// applies, else the phase's kernel sequence.
static std::vector<Launch> iteration_launches(const ampcg_ctx* c, int ph) {
  if (c->use_loop) return {c->loop[(c->fused_mask >> ph) & 1u][ph]};
  return c->seq[ph];
}

static cudaError_t launch_phase(ampcg_ctx* c, int ph, cudaStream_t s, cudaEvent_t* ev) {
  ArgPack pa(c, 1);
  int slot = -1;
  for (const Launch& L : iteration_launches(c, ph)) {
    while (ev && slot < L.slot) {   // slots without a kernel in this phase get an empty interval
      cudaError_t e = cudaEventRecord(ev[++slot], s);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = L.coop ? cudaLaunchCooperativeKernel(L.fn, dim3(L.grid), dim3(L.block), pa.args(L),
                                                         (size_t)L.smem, s)
                           : cudaLaunchKernel(L.fn, dim3(L.grid), dim3(L.block), pa.args(L), (size_t)L.smem, s);
    if (e != cudaSuccess) return e;
  }
  while (ev && slot < 4) {
    cudaError_t e = cudaEventRecord(ev[++slot], s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static cudaError_t add_kernel_node(cudaGraphNode_t* node, cudaGraph_t g, const cudaGraphNode_t* dep,
                                   const void* fn, int grid, int block, void** args, int smem = 0) {
  cudaKernelNodeParams p;
  memset(&p, 0, sizeof(p));
  p.func = (void*)fn;
  p.gridDim = dim3(grid);
  p.blockDim = dim3(block);
  p.sharedMemBytes = (unsigned)smem;
  p.kernelParams = args;
  p.extra = nullptr;
  return cudaGraphAddKernelNode(node, g, dep, dep ? 1 : 0, &p);
}

// Loop graph:
//   WHILE(!done) {
//     k_phase;                                  // SWITCH value = current pair
//     SWITCH { body ph (one per pair 2 u_z + u_r):
//       WHILE(pair == ph && !done) { `chunk` x (ph's launch sequence); k_chunk_ctl } }
//     k_loop_ctl }
// A SWITCH is evaluated once per precision change (about 5 us each on B300,
// against about 1.3 us per kernel node); after a change or the stop inside a
// chunk, the chunk's remaining launches return at entry (phase_mismatch,
// done).
static ampcg_status ensure_graph(ampcg_ctx* c, int chunk) {
  if (c->gexec && c->graph_chunk == chunk && c->graph_fused == c->fused_mask) return AMPCG_OK;
  if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
  if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
  CUDA_TRY(cudaGraphCreate(&c->graph, 0));
  cudaGraphConditionalHandle hw;
  CUDA_TRY(cudaGraphConditionalHandleCreate(&hw, c->graph, 1u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hw;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wnode;
  CUDA_TRY(cudaGraphAddNode(&wnode, c->graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaGraphConditionalHandle hs;
  CUDA_TRY(cudaGraphConditionalHandleCreate(&hs, body, AMPCG_PHASE_NONE, cudaGraphCondAssignDefault));
  DevState* st = c->st;
  void* aphase[2] = {&st, &hs};
  cudaGraphNode_t kphase;
  CUDA_TRY(add_kernel_node(&kphase, body, nullptr, (const void*)k_phase, 1, 1, aphase));
  cudaGraphNodeParams sp = {cudaGraphNodeTypeConditional};
  sp.type = cudaGraphNodeTypeConditional;
  sp.conditional.handle = hs;
  sp.conditional.type = cudaGraphCondTypeSwitch;
  sp.conditional.size = 6;
  cudaGraphNode_t snode;
  CUDA_TRY(cudaGraphAddNode(&snode, body, &kphase, nullptr, 1, &sp));
  ArgPack pa(c);
  for (int ph = 0; ph < 6; ++ph) {
    cudaGraph_t pg = sp.conditional.phGraph_out[ph];
    cudaGraphConditionalHandle hi;
    CUDA_TRY(cudaGraphConditionalHandleCreate(&hi, pg, 1u, cudaGraphCondAssignDefault));
    cudaGraphNodeParams ip = {cudaGraphNodeTypeConditional};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hi;
    ip.conditional.type = cudaGraphCondTypeWhile;
    ip.conditional.size = 1;
    cudaGraphNode_t inode;
    CUDA_TRY(cudaGraphAddNode(&inode, pg, nullptr, nullptr, 0, &ip));
    cudaGraph_t ib = ip.conditional.phGraph_out[0];
    cudaGraphNode_t kn = nullptr;
    // k_loop runs the whole chunk in one launch
    const std::vector<Launch> seq = iteration_launches(c, ph);
    pa.iters = chunk;
    for (int i = 0; i < (c->use_loop ? 1 : chunk); ++i)
      for (const Launch& L : seq) {
        cudaGraphNode_t nn;
        CUDA_TRY(add_kernel_node(&nn, ib, kn ? &kn : nullptr, L.fn, L.grid, L.block, pa.args(L), L.smem));
        if (L.coop) {
          cudaLaunchAttributeValue av;
          memset(&av, 0, sizeof(av));
          av.cooperative = 1;
          CUDA_TRY(cudaGraphKernelNodeSetAttribute(nn, cudaLaunchAttributeCooperative, &av));
        }
        kn = nn;
      }
    int phv = ph;
    void* actl[3] = {&st, &hi, &phv};
    cudaGraphNode_t cn;
    CUDA_TRY(add_kernel_node(&cn, ib, kn ? &kn : nullptr, (const void*)k_chunk_ctl, 1, 1, actl));
  }
  void* actl[2] = {&st, &hw};
  cudaGraphNode_t cnode;
  CUDA_TRY(add_kernel_node(&cnode, body, &snode, (const void*)k_loop_ctl, 1, 1, actl));
  CUDA_TRY(cudaGraphInstantiate(&c->gexec, c->graph, 0));
  c->graph_chunk = chunk;
  c->graph_fused = c->fused_mask;
  return AMPCG_OK;
}

static ampcg_status check_policy(const ampcg_policy* p) {
  if (p->u0 < 0 || p->u0 > 2 || p->fixed_uz < 0 || p->fixed_uz > 2 || p->fixed_ur < 0 ||
      p->fixed_ur > 1)
    return fail(AMPCG_ERR_INVALID_ARG, "precision codes: u0/fixed_uz in {0,1,2}, fixed_ur in {0,1}");
  if (p->criterion < 0 || p->criterion > 2) return fail(AMPCG_ERR_INVALID_ARG, "bad criterion");
  if (p->scale < 0 || p->scale > 3) return fail(AMPCG_ERR_INVALID_ARG, "bad scale mode");
  if (p->d < 0 || p->ell < 1 || p->d > kRing - 2 || p->ell > kRing - 1)
    return fail(AMPCG_ERR_INVALID_ARG, "need 0 <= d <= %d and 1 <= ell <= %d", kRing - 2, kRing - 1);
  if (p->verify_refresh < 0 || p->graph_chunk < 0)
    return fail(AMPCG_ERR_INVALID_ARG, "verify_refresh and graph_chunk must be >= 0");
  return AMPCG_OK;
}

static void init_state(DevState* h, const ampcg_policy* p, double tol, int maxit, ampcg_ctx* c) {
  memset(h, 0, sizeof(*h));
  h->maxit = maxit;
  h->criterion = p->criterion;
  h->u0 = p->u0;
  h->d = p->d;
  h->ell = p->ell;
  h->scale = p->scale;
  h->latch = p->latch;
  h->fixed_uz = p->fixed_uz;
  h->fixed_ur = p->fixed_ur;
  h->C = p->C;
  h->tau_zs = p->tau_zs;
  h->tau_zh = p->tau_zh;
  h->tol = tol;
  h->uz = (p->criterion == AMPCG_CRIT_FIXED) ? p->fixed_uz : p->u0;
  h->ur = P64;
  h->uz_p = h->uz;
  h->first = 1;
  h->k_body = -1;
  h->switch_iter[0] = h->switch_iter[1] = h->switch_iter[2] = -1;
  h->delta_hist = c ? c->dhist : nullptr;
  h->prec_hist = c ? c->phist : nullptr;
}

// Launch-by-launch loop with a CUDA event pair around every iteration kernel
// (timing mode).  The host reads the state after each iteration to pick the
// next phase's kernels; an iteration counts when it advanced the counter.
static ampcg_status timed_loop(ampcg_ctx* c, ampcg_kernel_times* kt, cudaEvent_t* ev,
                               long long& launches) {
  cudaStream_t s = c->stream;
  while (!c->hst->done) {
    int k0 = c->hst->k;
    int ph = 2 * c->hst->uz + c->hst->ur;
    if (ph < 0 || ph > 5) return fail(AMPCG_ERR_CUDA, "invalid phase %d in device state", ph);
    CUDA_TRY(launch_phase(c, ph, s, ev));
    const std::vector<Launch> seq = iteration_launches(c, ph);
    launches += (long long)seq.size();
    CUDA_TRY(cudaMemcpyAsync(c->hst, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (c->hst->k > k0) {
      for (int j = 0; j < 4; ++j) {
        bool has = false;
        for (const Launch& L : seq) has = has || L.slot == j;
        if (!has) continue;
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, ev[j], ev[j + 1]));
        kt->ms[j][ph] += ms;
        kt->launches[j][ph] += 1;
      }
    }
  }
  return AMPCG_OK;
}

// Tuning slot of a scale mode: the iteration kernel's form is chosen
// separately for NONE, the lagged and the exact power of two (-1: L2, which
// has the four-barrier form only).
static int scale_slot(int scale) {
  if (scale == AMPCG_SCALE_NONE) return 0;
  if (scale == AMPCG_SCALE_LINF_POW2_LAG) return 1;
  if (scale == AMPCG_SCALE_LINF_POW2) return 2;
  return -1;
}

static ampcg_status solve_impl(ampcg_ctx* c, const double* b, double* x, double tol, int maxit,
                               const ampcg_policy* policy, ampcg_result* res,
                               ampcg_kernel_times* kt, cudaStream_t s_override = nullptr);

extern "C" ampcg_status ampcg_solve(ampcg_t c, const double* b, double* x, double tol, int maxit,
                                    const ampcg_policy* policy, ampcg_result* res) {
  return solve_impl(c, b, x, tol, maxit, policy, res, nullptr);
}

extern "C" ampcg_status ampcg_solve_timed(ampcg_t c, const double* b, double* x, double tol,
                                          int maxit, const ampcg_policy* policy, ampcg_result* res,
                                          ampcg_kernel_times* kt) {
  if (!kt) return fail(AMPCG_ERR_INVALID_ARG, "NULL kernel-times output");
  memset(kt, 0, sizeof(*kt));
  return solve_impl(c, b, x, tol, maxit, policy, res, kt);
}

static ampcg_status solve_impl(ampcg_ctx* c, const double* b, double* x, double tol, int maxit,
                               const ampcg_policy* policy, ampcg_result* res,
                               ampcg_kernel_times* kt, cudaStream_t s_override) {
  auto t0 = std::chrono::steady_clock::now();
  if (!c) return fail(AMPCG_ERR_INVALID_ARG, "NULL context");
  if (!b || !x) return fail(AMPCG_ERR_INVALID_ARG, "NULL b or x");
  if (!(tol > 0.0) || maxit < 0) return fail(AMPCG_ERR_INVALID_ARG, "need tol > 0, maxit >= 0");
  ampcg_policy pol;
  if (policy) pol = *policy;
  else ampcg_policy_default(&pol);
  ampcg_status ps = check_policy(&pol);
  if (ps != AMPCG_OK) return ps;
  if (pol.scale == AMPCG_SCALE_LINF_POW2_LAG && c->mtype == M_CHEBYSHEV)
    return fail(AMPCG_ERR_UNSUPPORTED, "the lagged scale is not offered with the Chebyshev preconditioner "
                "(use AMPCG_SCALE_LINF_POW2)");
  // default chunk: long for the persistent kernel (a launch ends at the stop
  // or a precision change anyway; 256 measured 0.8 ms faster than 16 on the
  // 128^3 solves), short for the kernel sequence (its launches after the stop
  // return at entry but still cost a launch each)
  int chunk = pol.graph_chunk > 0 ? pol.graph_chunk : (c->use_loop ? kLoopChunk : kSeqChunk);
  // the persistent kernel's three-barrier form, per pair as tuned
  // (automatic: three): for the scale modes whose omega_{k+1} is known before
  // delta_{k+1} is reduced, and for the exact power of two, whose z_{k+1} is
  // formed with the exponent of max|r_k| and kept when max|r_{k+1}| has it
  c->fused_mask = 0;
  const int fslot = scale_slot(pol.scale);
  if (fslot >= 0) {
    const int* form = c->loop_form[fslot];
    for (int ph = 0; ph < 6; ++ph)
      if (form[ph] != 0) c->fused_mask |= 1u << ph;
  }
  cudaSetDevice(c->device);
  cudaStream_t s = s_override ? s_override : c->stream;
  ampcg_status hs = ensure_hist(c, maxit);
  if (hs != AMPCG_OK) return hs;
  bool b_dev = is_device_ptr(b), x_dev = is_device_ptr(x);
  size_t vb = (size_t)c->n * sizeof(double);
  CUDA_TRY(cudaMemcpyAsync(c->b, b, vb, b_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(c->x, x, vb, x_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  init_state(c->hst, &pol, tol, maxit, c);
  CUDA_TRY(cudaMemcpyAsync(c->st, c->hst, sizeof(DevState), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemsetAsync(c->bar, 0, 12 * sizeof(GridSumBarrier), s));
  if (!kt) {
    hs = ensure_graph(c, chunk);
    if (hs != AMPCG_OK) return hs;
  }
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t e_first = nullptr, e_last = nullptr;
  struct EvGuard {
    cudaEvent_t* ev; cudaEvent_t* a; cudaEvent_t* b;
    ~EvGuard() {
      for (int i = 0; i < 5; ++i) if (ev[i]) cudaEventDestroy(ev[i]);
      if (*a) cudaEventDestroy(*a);
      if (*b) cudaEventDestroy(*b);
    }
  } guard{ev, &e_first, &e_last};
  if (kt) {
    for (int i = 0; i < 5; ++i) CUDA_TRY(cudaEventCreate(&ev[i]));
    CUDA_TRY(cudaEventCreate(&e_first));
    CUDA_TRY(cudaEventCreate(&e_last));
  }
  Sell A = c->sell();
  Bufs B = c->bufs();
  int64_t rows_pad = c->nslices * 32;
  int gi = occ_grid(c->idx16 ? (const void*)k_init<1> : (const void*)k_init<0>, 148, rows_pad);
  if (gi > c->g_max) gi = c->g_max;
  if (c->idx16) k_init<1><<<gi, kBlock, 0, s>>>(A, B, c->st);
  else k_init<0><<<gi, kBlock, 0, s>>>(A, B, c->st);
  CUDA_TRY(cudaGetLastError());
  long long launches = 1;  // k_init
  int runs_before[6] = {0, 0, 0, 0, 0, 0};
  int loops_before = 0;
  if (kt) {
    CUDA_TRY(cudaEventRecord(e_first, s));
    CUDA_TRY(cudaMemcpyAsync(c->hst, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  for (;;) {
    if (kt) {
      ampcg_status ts = timed_loop(c, kt, ev, launches);
      if (ts != AMPCG_OK) return ts;
    } else {
      CUDA_TRY(cudaGraphLaunch(c->gexec, s));
    }
    launches += 1;  // true residual
    if (c->idx16) k_true_residual<1><<<c->g_rows, kBlock, 0, s>>>(A, B, c->st);
    else k_true_residual<0><<<c->g_rows, kBlock, 0, s>>>(A, B, c->st);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(c->hst, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    const DevState& h = *c->hst;
    if (!kt) {
      // device loop: every outer body launches k_phase and k_loop_ctl, every
      // inner chunk its pair's sequence `chunk` times and k_chunk_ctl (the
      // launches that return at entry after a change or the stop included)
      launches += 2LL * (h.loop_runs - loops_before);
      loops_before = h.loop_runs;
      for (int ph = 0; ph < 6; ++ph) {
        const long long per_chunk = c->use_loop ? 1 : (long long)chunk * (long long)c->seq[ph].size();
        launches += (per_chunk + 1) * (h.chunk_runs[ph] - runs_before[ph]);
        runs_before[ph] = h.chunk_runs[ph];
      }
    }
    // reading R9: verify, and replace r when the true residual misses tol
    bool refresh = h.status == ST_OK && h.refreshes < pol.verify_refresh && h.k < maxit &&
                   h.true_relres * h.nb > h.tol_nb;
    if (!refresh) break;
    k_refresh<<<c->g_elem, kBlock, 0, s>>>(B, c->n, c->st);
    CUDA_TRY(cudaGetLastError());
    launches += 1;
    if (kt) {
      CUDA_TRY(cudaMemcpyAsync(c->hst, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaStreamSynchronize(s));
    }
  }
  if (kt) {
    CUDA_TRY(cudaEventRecord(e_last, s));
    CUDA_TRY(cudaEventSynchronize(e_last));
    float tot = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&tot, e_first, e_last));
    kt->total_ms = tot;
  }
  const DevState& h = *c->hst;
  CUDA_TRY(cudaMemcpyAsync(x, c->x, vb, x_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  int iters = h.k;
  if (res) {
    if (res->relres_hist)   // delta_k, divided by ||b|| below
      CUDA_TRY(cudaMemcpyAsync(res->relres_hist, c->dhist, (iters + 1) * sizeof(double),
                               cudaMemcpyDeviceToHost, s));
    if (res->prec_hist && iters > 0)
      CUDA_TRY(cudaMemcpyAsync(res->prec_hist, c->phist, iters, cudaMemcpyDeviceToHost, s));
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  ampcg_status st = (ampcg_status)h.status;
  if (res) {
    res->iters = iters;
    res->converged = h.status == ST_OK;
    res->refreshes = h.refreshes;
    res->status = h.status;
    res->true_relres = h.true_relres;
    res->updated_relres = h.delta / h.nb;
    if (res->relres_hist)
      for (int i = 0; i <= iters; ++i) res->relres_hist[i] /= h.nb;
    for (int i = 0; i < 3; ++i) res->switch_iter[i] = h.switch_iter[i];
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    res->kernel_launches = launches;
  }
  if (h.status == ST_INTERNAL) {
    st = AMPCG_ERR_CUDA;
    if (res) res->status = st;
    return fail(st, "internal error: device loop made no progress or ran a kernel for the wrong "
                "precision pair (iteration %d)", iters);
  }
  if (h.status == ST_TIMEOUT)
    return fail(AMPCG_ERR_TIMEOUT, "a grid-barrier wait of the iteration kernel ran out at iteration %d "
                "(a block never arrived)", iters);
  if (st != AMPCG_OK && st != AMPCG_NOT_CONVERGED)
    fail(st, "solve stopped at iteration %d: %s", iters, ampcg_status_string(st));
  return st;
}

// ---------------------------------------------------------------------------
// step entry points

extern "C" ampcg_status ampcg_spmv(ampcg_t c, int prec, const void* p, void* q) {
  if (!c || !p || !q) return fail(AMPCG_ERR_INVALID_ARG, "NULL argument");
  Sell A = c->sell();
  cudaStream_t s = c->stream;
  if (prec == AMPCG_FP64) {
    if (c->idx16) k_spmv_step<P64, 1><<<c->g_rows, kBlock, 0, s>>>(A, p, q);
    else k_spmv_step<P64, 0><<<c->g_rows, kBlock, 0, s>>>(A, p, q);
  } else if (prec == AMPCG_FP32) {
    if (c->idx16) k_spmv_step<P32, 1><<<c->g_rows, kBlock, 0, s>>>(A, p, q);
    else k_spmv_step<P32, 0><<<c->g_rows, kBlock, 0, s>>>(A, p, q);
  } else {
    return fail(AMPCG_ERR_INVALID_ARG, "spmv precision must be FP64 or FP32");
  }
  CUDA_TRY(cudaGetLastError());
  return AMPCG_OK;
}

template <int UZ, int UR, int IT>
static cudaError_t launch_spmv_loop_step(ampcg_ctx* c, const Bufs& B) {
  const void* fn = loop_spmv_kernel(UZ, UR, IT);
  const int smem = LoopStageCfg<UR, IT>::kBytes;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  Sell A = c->sell();
  Bufs Bc = B;
  DevState* st = c->st;
  void* args[3] = {&A, &Bc, &st};
  return cudaLaunchKernel(fn, dim3(c->loop[0][2 * UZ + UR].grid), dim3(kLoopBlock), args, (size_t)smem, c->stream);
}

template <int UZ, int UR>
static cudaError_t spmv_loop_step_t(ampcg_ctx* c, const Bufs& B) {
  return c->idx16 ? launch_spmv_loop_step<UZ, UR, 1>(c, B) : launch_spmv_loop_step<UZ, UR, 0>(c, B);
}

extern "C" ampcg_status ampcg_spmv_loop_step(ampcg_t c, int uz, int ur, const void* p, void* q,
                                             double* gamma) {
  if (!c || !p || !q) return fail(AMPCG_ERR_INVALID_ARG, "NULL argument");
  if (uz < 0 || uz > 2 || ur < 0 || ur > 1) return fail(AMPCG_ERR_INVALID_ARG, "bad precision");
  if (!c->use_loop)
    return fail(AMPCG_ERR_UNSUPPORTED, "the context does not run the persistent iteration kernel "
                "(Chebyshev preconditioner or slices wider than %d)", kStageW);
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  Bufs B = c->bufs();
  B.p[0] = const_cast<void*>(p);
  B.p[1] = const_cast<void*>(p);
  B.q = q;
  cudaError_t e;
  if (uz == P64) e = ur == P64 ? spmv_loop_step_t<P64, P64>(c, B) : spmv_loop_step_t<P64, P32>(c, B);
  else if (uz == P32) e = ur == P64 ? spmv_loop_step_t<P32, P64>(c, B) : spmv_loop_step_t<P32, P32>(c, B);
  else e = ur == P64 ? spmv_loop_step_t<P16, P64>(c, B) : spmv_loop_step_t<P16, P32>(c, B);
  CUDA_TRY(e);
  const int G = c->loop[0][2 * uz + ur].grid;
  std::vector<double> part((size_t)G);
  CUDA_TRY(cudaMemcpyAsync(part.data(), c->part, (size_t)G * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (gamma) {
    double g = 0.0;
    for (int i = 0; i < G; ++i) g += part[(size_t)i];
    *gamma = g;
  }
  return AMPCG_OK;
}

extern "C" ampcg_status ampcg_spmv_block(ampcg_t c, int prec, const void* p, void* q) {
  if (!c || !p || !q) return fail(AMPCG_ERR_INVALID_ARG, "NULL argument");
  if (prec != AMPCG_FP64 && prec != AMPCG_FP32) return fail(AMPCG_ERR_INVALID_ARG, "block spmv precision must be FP64 or FP32");
  if (!c->bs3) return fail(AMPCG_ERR_UNSUPPORTED, "the context has no 3 x 3 block layout");
  BSell A = c->bsell();
  void* args[3] = {&A, const_cast<void**>(&p), &q};
  const void* fn = bsr_spmv_step_kernel(prec);
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const int grid = occ_grid(fn, sms, c->nbs3 * 32);
  CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(kBlock), args, 0, c->stream));
  return AMPCG_OK;
}

extern "C" ampcg_status ampcg_residual(ampcg_t c, const double* b, const double* x, double* r) {
  if (!c || !b || !x || !r) return fail(AMPCG_ERR_INVALID_ARG, "NULL argument");
  Sell A = c->sell();
  if (c->idx16) k_residual_step<1><<<c->g_rows, kBlock, 0, c->stream>>>(A, b, x, r);
  else k_residual_step<0><<<c->g_rows, kBlock, 0, c->stream>>>(A, b, x, r);
  CUDA_TRY(cudaGetLastError());
  return AMPCG_OK;
}

template <int UZ, int UR>
static void launch_precond_step(ampcg_ctx* c, const Bufs& B, const DevState* st) {
  if (c->mtype == M_NONE) k_precond_step<UZ, UR, M_NONE><<<c->g_elem, kBlock, 0, c->stream>>>(B, c->n, st);
  else k_precond_step<UZ, UR, M_JACOBI><<<c->g_elem, kBlock, 0, c->stream>>>(B, c->n, st);
}

extern "C" ampcg_status ampcg_precond_apply(ampcg_t c, int uz, int ur, double omega, const void* r,
                                            void* z) {
  if (!c || !r || !z) return fail(AMPCG_ERR_INVALID_ARG, "NULL argument");
  if (uz < 0 || uz > 2 || ur < 0 || ur > 1) return fail(AMPCG_ERR_INVALID_ARG, "bad precision");
  if (!(omega != 0.0) || !std::isfinite(omega)) return fail(AMPCG_ERR_INVALID_ARG, "omega must be finite, nonzero");
  // a private state block carries omega; the step does no storage conversion
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  DevState* h = c->hst;
  ampcg_policy dp;
  ampcg_policy_default(&dp);
  init_state(h, &dp, 1.0, 0, nullptr);
  h->omega = omega;
  h->omega_f = (float)omega;
  int E;
  double f = std::frexp(omega, &E);
  h->omega_pow2 = (f == 0.5 || f == -0.5) && omega > 0;
  h->omega_e = E - 1;
  h->uz = uz;
  h->ur = ur;
  CUDA_TRY(cudaMemcpyAsync(c->st, h, sizeof(DevState), cudaMemcpyHostToDevice, c->stream));
  Bufs B = c->bufs();
  B.r64 = (double*)r;
  B.r32 = (float*)r;
  B.z = z;
  if (c->mtype == M_CHEBYSHEV) {
    // the precondition part of the phase's launch sequence on the caller's r, z
    ArgPack pa(c);
    pa.B = B;
    for (const Launch& L : c->seq[2 * uz + ur]) {
      if (L.slot != 0) break;
      CUDA_TRY(cudaLaunchKernel(L.fn, dim3(L.grid), dim3(kBlock), pa.args(L), (size_t)L.smem, c->stream));
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return AMPCG_OK;
  }
  if (ur == P64) {
    if (uz == P64) launch_precond_step<P64, P64>(c, B, c->st);
    else if (uz == P32) launch_precond_step<P32, P64>(c, B, c->st);
    else launch_precond_step<P16, P64>(c, B, c->st);
  } else {
    if (uz == P64) launch_precond_step<P64, P32>(c, B, c->st);
    else if (uz == P32) launch_precond_step<P32, P32>(c, B, c->st);
    else launch_precond_step<P16, P32>(c, B, c->st);
  }
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return AMPCG_OK;
}

// Longest residual-norm sequence ampcg_selector_trace replays: delta[0..m]
// with m < kTraceMax, so (m + 1) * sizeof(double) cannot overflow.
constexpr int kTraceMax = 1 << 28;

extern "C" ampcg_status ampcg_selector_trace(const ampcg_policy* policy, const double* delta,
                                             int m, double nb, double tol, uint8_t* out) {
  if (!policy || !delta || !out || m < 0) return fail(AMPCG_ERR_INVALID_ARG, "bad argument");
  if (m > kTraceMax - 1)
    return fail(AMPCG_ERR_INVALID_ARG, "selector replay takes at most %d residual norms (m <= %d); got m = %d",
                kTraceMax, kTraceMax - 1, m);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(AMPCG_ERR_NO_DEVICE, "no CUDA device visible");
  }
  ampcg_status ps = check_policy(policy);
  if (ps != AMPCG_OK) return ps;
  double* d_delta = nullptr;
  unsigned char* d_out = nullptr;
  unsigned char* d_ph = nullptr;
  DevState* d_st = nullptr;
  DevState h;
  init_state(&h, policy, tol, m + 1, nullptr);
  h.nb = nb;
  h.tol_nb = tol * nb;
  h.maxr = 1.0;
  const size_t cnt = (size_t)m + 1;
  cudaError_t e = cudaMalloc(&d_delta, cnt * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_out, cnt);
  if (e == cudaSuccess) e = cudaMalloc(&d_ph, cnt);
  if (e == cudaSuccess) e = cudaMalloc(&d_st, sizeof(DevState));
  if (e == cudaSuccess) {
    h.delta_hist = d_delta;
    h.prec_hist = d_ph;
    e = cudaMemcpy(d_delta, delta, cnt * sizeof(double), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemcpy(d_st, &h, sizeof(DevState), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_selector_trace<<<1, 32>>>(d_st, m, d_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, d_out, cnt, cudaMemcpyDeviceToHost);
  cudaFree(d_delta);
  cudaFree(d_out);
  cudaFree(d_ph);
  cudaFree(d_st);
  if (e != cudaSuccess) return fail(AMPCG_ERR_CUDA, "selector trace: %s", cudaGetErrorString(e));
  return AMPCG_OK;
}

// ---------------------------------------------------------------------------
// Selector replay without any device allocation.
//
// ampcg_selector_trace above allocates its device scratch (the state block,
// the residual history and two byte arrays) with cudaMalloc on every call.
// This variant keeps that scratch in one file-scope device array instead, so
// callers that must not allocate device memory can use it.  Every GPU that
// loads the library holds the array (kNoAllocTraceBytes) until process exit.
// Host code cannot use the array's name as a device address: the address is
// looked up with cudaGetSymbolAddress on the first call made in a device's
// context (that device current) and cached together with the context's
// identity, so a call in a later context of the device (after a reset of its
// primary context) looks the address up again instead of using a stale one.

namespace {

constexpr int kNoAllocTraceMax = 65536;  // entries delta[0..m], i.e. m + 1 <= this

struct NoAllocTraceScratch {
  DevState st;
  double delta[kNoAllocTraceMax];
  unsigned char prec[kNoAllocTraceMax];
  unsigned char out[kNoAllocTraceMax];
};

constexpr size_t kNoAllocTraceBytes = sizeof(NoAllocTraceScratch);

static __device__ __align__(256) unsigned char g_noalloc_trace_scratch[kNoAllocTraceBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
struct NoAllocSlot {
  unsigned long long ctx_id;  // identity of the context the address belongs to
  void* addr;
};
NoAllocSlot g_noalloc[kMaxDevices] = {};

// Identity of the calling thread's current context (driver entry points
// resolved through the runtime, so the library does not link the driver
// library itself).  False when there is no current context or the driver
// cannot tell; the caller then does not reuse a cached address.
typedef CUresult (*PfnCtxGetCurrent)(CUcontext*);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long*);
bool current_ctx_id(unsigned long long* id) {
  static std::once_flag once;
  static PfnCtxGetCurrent get_cur = nullptr;
  static PfnCtxGetId get_id = nullptr;
  std::call_once(once, []() {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = (PfnCtxGetCurrent)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (PfnCtxGetId)f;
    cudaGetLastError();
  });
  if (!get_cur || !get_id) return false;
  CUcontext ctx = nullptr;
  if (get_cur(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of the scratch array in the current device's context: looked
// up once per context (with that device current) and cached.
ampcg_status noalloc_scratch(NoAllocTraceScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(AMPCG_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(AMPCG_ERR_UNSUPPORTED, "device index %d too large", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  unsigned long long id = 0;
  NoAllocSlot& slot = g_noalloc[dev];
  if (slot.addr && current_ctx_id(&id) && id == slot.ctx_id) {
    *out = (NoAllocTraceScratch*)slot.addr;
    return AMPCG_OK;
  }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_trace_scratch);   // makes the device's context current if needed
  if (e != cudaSuccess || !p)
    return fail(AMPCG_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
  if (current_ctx_id(&id)) {
    slot.ctx_id = id;
    slot.addr = p;
  } else {
    slot.addr = nullptr;   // identity unknown: look the address up on every call
  }
  *out = (NoAllocTraceScratch*)p;
  return AMPCG_OK;
}

}  // namespace

extern "C" ampcg_status ampcg_selector_trace_noalloc(const ampcg_policy* policy,
                                                     const double* delta, int m, double nb,
                                                     double tol, uint8_t* out) {
  if (!policy || !delta || !out || m < 0) return fail(AMPCG_ERR_INVALID_ARG, "bad argument");
  if (m > kNoAllocTraceMax - 1)
    return fail(AMPCG_ERR_INVALID_ARG,
                "selector replay without allocation takes at most %d residual norms (m <= %d); got m = %d",
                kNoAllocTraceMax, kNoAllocTraceMax - 1, m);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(AMPCG_ERR_NO_DEVICE, "no CUDA device visible");
  }
  ampcg_status ps = check_policy(policy);
  if (ps != AMPCG_OK) return ps;
  NoAllocTraceScratch* sc = nullptr;
  ps = noalloc_scratch(&sc);
  if (ps != AMPCG_OK) return ps;
  // Everything the kernel reads is written here first: the whole state block
  // (zeroed fields included) and delta[0..m]; prec[k] and out[k] are written
  // by the kernel before they are read.  Entries past m keep the previous
  // call's contents and are never read.
  DevState h;
  init_state(&h, policy, tol, m + 1, nullptr);
  h.nb = nb;
  h.tol_nb = tol * nb;
  h.maxr = 1.0;
  h.delta_hist = sc->delta;
  h.prec_hist = sc->prec;
  cudaError_t e = cudaMemcpy(sc->delta, delta, (size_t)(m + 1) * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(&sc->st, &h, sizeof(DevState), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_selector_trace<<<1, 32>>>(&sc->st, m, sc->out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, sc->out, (size_t)(m + 1), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(AMPCG_ERR_CUDA, "selector trace (no allocation): %s", cudaGetErrorString(e));
  return AMPCG_OK;
}


// ---------------------------------------------------------------------------
// Failure detection of the grid barriers without a GPU fault: one barrier of
// the kind the persistent iteration kernel uses, with a short caller-given
// poll limit, optionally with one block that never arrives.

extern "C" ampcg_status ampcg_barrier_check(int nblocks, int absent_block, long long spin_limit) {
  if (nblocks < 2 || nblocks > 64) return fail(AMPCG_ERR_INVALID_ARG, "nblocks must be in [2, 64]");
  if (absent_block < -1 || absent_block >= nblocks)
    return fail(AMPCG_ERR_INVALID_ARG, "absent_block must be -1 or in [0, nblocks)");
  if (spin_limit < 1 || spin_limit > kBarrierSpin)
    return fail(AMPCG_ERR_INVALID_ARG, "spin_limit must be in [1, %lld]", kBarrierSpin);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(AMPCG_ERR_NO_DEVICE, "no CUDA device visible");
  }
  int coop = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) return fail(AMPCG_ERR_UNSUPPORTED, "device has no cooperative launch");
  GridSumBarrier* g = nullptr;
  double* part = nullptr;
  int* out = nullptr;
  cudaError_t e = cudaMalloc(&g, sizeof(GridSumBarrier));
  if (e == cudaSuccess) e = cudaMalloc(&part, 4 * (size_t)nblocks * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&out, (size_t)nblocks * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(g, 0, sizeof(GridSumBarrier));
  if (e == cudaSuccess) e = cudaMemset(out, 0, (size_t)nblocks * sizeof(int));
  std::vector<int> h(nblocks, 0);
  if (e == cudaSuccess) {
    void* args[5] = {&g, &part, &absent_block, &spin_limit, &out};
    e = cudaLaunchCooperativeKernel((const void*)k_barrier_check, dim3(nblocks), dim3(256), args, 0, nullptr);
  }
  if (e == cudaSuccess) e = cudaMemcpy(h.data(), out, (size_t)nblocks * sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(g);
  cudaFree(part);
  cudaFree(out);
  if (e != cudaSuccess) return fail(AMPCG_ERR_CUDA, "barrier check: %s", cudaGetErrorString(e));
  int passed = 0, timed_out = 0;
  for (int b = 0; b < nblocks; ++b) {
    if (h[b] == 1) ++passed;
    else if (h[b] == 0) ++timed_out;
  }
  if (timed_out > 0)
    return fail(AMPCG_ERR_TIMEOUT, "grid barrier: %d of %d arriving blocks gave up after %lld polls",
                timed_out, passed + timed_out, spin_limit);
  return AMPCG_OK;
}

// ---------------------------------------------------------------------------
// New values on the same pattern, and the adjoint solve.

// Block-row layout of a 3 x 3 block matrix (bsr.cuh): values (and the
// Chebyshev Ahat copies) from the scalar sliced layout, after creation and
// after every value change.
static ampcg_status fill_block_layout(ampcg_ctx* c) {
  if (!c->bs3) return AMPCG_OK;
  const int gb = (int)((c->nbs3 * 32 + kBlock - 1) / kBlock);
  const bool ch = c->mtype == M_CHEBYSHEV;
  if (c->idx16)
    k_bfill<1><<<gb, kBlock, 0, c->stream>>>(c->sell(), c->rowptr, c->bsell(), c->bcol3, c->bv64, c->bv32,
                                             ch ? c->ah64 : nullptr, ch ? c->bah64 : nullptr, c->bah32, c->bah16);
  else
    k_bfill<0><<<gb, kBlock, 0, c->stream>>>(c->sell(), c->rowptr, c->bsell(), c->bcol3, c->bv64, c->bv32,
                                             ch ? c->ah64 : nullptr, ch ? c->bah64 : nullptr, c->bah32, c->bah16);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return AMPCG_OK;
}

static ampcg_status build_block_layout(ampcg_ctx* c) {
  cudaStream_t s = c->stream;
  c->nb3 = c->n / 3;
  c->nbs3 = (c->nb3 + 31) / 32;
  long long* total = nullptr;
  ampcg_status st;
  if ((st = dalloc(&c->bw, c->nbs3)) != AMPCG_OK) return st;
  if ((st = dalloc(&c->boff, c->nbs3)) != AMPCG_OK) return st;
  if ((st = dalloc(&total, 2)) != AMPCG_OK) return st;
  const int gs = (int)((c->nbs3 + kBlock - 1) / kBlock);
  k_bslice_width<<<gs, kBlock, 0, s>>>(c->nb3, c->nbs3, c->rowptr, c->bw);
  k_slice_offsets<<<1, 1024, 0, s>>>(c->nbs3, c->bw, c->boff, total);
  long long tot2[2] = {0, 0};
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(tot2, total, sizeof(tot2), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(total);
  if (e != cudaSuccess) return fail(AMPCG_ERR_CUDA, "block layout: %s", cudaGetErrorString(e));
  c->bstored = tot2[0];
  if ((st = dalloc(&c->bcol3, c->bstored)) != AMPCG_OK) return st;
  if ((st = dalloc(&c->bv64, 9 * c->bstored)) != AMPCG_OK) return st;
  if ((st = dalloc(&c->bv32, 9 * c->bstored)) != AMPCG_OK) return st;
  if (c->mtype == M_CHEBYSHEV) {
    if ((st = dalloc(&c->bah64, 9 * c->bstored)) != AMPCG_OK) return st;
    if ((st = dalloc(&c->bah32, 9 * c->bstored)) != AMPCG_OK) return st;
    if ((st = dalloc(&c->bah16, 9 * c->bstored)) != AMPCG_OK) return st;
  }
  c->bs3 = true;
  if ((st = fill_block_layout(c)) != AMPCG_OK) return st;
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  if ((st = build_sequences(c, sms)) != AMPCG_OK) return st;
  if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
  if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
  // the block kernels' grids must fit the per-block partial arrays
  int gmax = c->g_max;
  for (int ph = 0; ph < 6; ++ph)
    for (const Launch& L : c->seq[ph]) gmax = L.grid > gmax ? L.grid : gmax;
  if (gmax > c->g_max) {
    cudaFree(c->part);
    cudaFree(c->pmax);
    c->part = nullptr;
    c->pmax = nullptr;
    c->g_max = gmax;
    if ((st = dalloc(&c->part, (size_t)c->g_max * 6)) != AMPCG_OK) return st;
    if ((st = dalloc(&c->pmax, (size_t)c->g_max * 2)) != AMPCG_OK) return st;
  }
  return AMPCG_OK;
}

// After new matrix values: the Chebyshev data follow A; with an automatic
// interval the constants change, so the launch sequences and the loop graph
// are rebuilt.
static ampcg_status refresh_precond(ampcg_ctx* c) {
  if (c->mtype != M_CHEBYSHEV) return AMPCG_OK;
  ampcg_status st = cheb_prepare(c);
  if (st != AMPCG_OK) return st;
  if (c->cheb_auto) {
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    if ((st = build_sequences(c, sms)) != AMPCG_OK) return st;
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
  }
  return AMPCG_OK;
}

extern "C" ampcg_status ampcg_precond_interval(ampcg_t c, double* lmin, double* lmax) {
  if (!c || !lmin || !lmax) return fail(AMPCG_ERR_INVALID_ARG, "NULL argument");
  if (c->mtype != M_CHEBYSHEV) return fail(AMPCG_ERR_INVALID_ARG, "not a Chebyshev preconditioner");
  *lmin = c->cheb_lmin;
  *lmax = c->cheb_lmax;
  return AMPCG_OK;
}

extern "C" ampcg_status ampcg_update_values(ampcg_t c, const double* vals) {
  if (!c || !vals) return fail(AMPCG_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = c->stream;
  const double* d_v = vals;
  double* t_v = nullptr;
  int* flags = nullptr;
  ampcg_status st = AMPCG_OK;
  if (!is_device_ptr(vals)) {
    if ((st = dalloc(&t_v, c->nnz)) != AMPCG_OK) return st;
    cudaError_t e = cudaMemcpyAsync(t_v, vals, c->nnz * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { cudaFree(t_v); return fail(AMPCG_ERR_CUDA, "copy: %s", cudaGetErrorString(e)); }
    d_v = t_v;
  }
  if ((st = dalloc(&flags, 1)) != AMPCG_OK) { if (t_v) cudaFree(t_v); return st; }
  int hf = 0;
  cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(int), s);
  Sell A = c->sell();
  if (e == cudaSuccess) {
    if (c->idx16)
      k_update_vals<1><<<c->g_rows, kBlock, 0, s>>>(A, c->rowptr, d_v, c->v64, c->v32, c->dinv64, c->dinv32, c->dinv16, flags);
    else
      k_update_vals<0><<<c->g_rows, kBlock, 0, s>>>(A, c->rowptr, d_v, c->v64, c->v32, c->dinv64, c->dinv32, c->dinv16, flags);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (t_v) cudaFree(t_v);
  cudaFree(flags);
  if (e != cudaSuccess) return fail(AMPCG_ERR_CUDA, "update values: %s", cudaGetErrorString(e));
  if (hf & 8) return fail(AMPCG_ERR_NONFINITE, "matrix has non-finite values (context now holds them)");
  if (hf & 4) return fail(AMPCG_ERR_NOT_SPD, "a diagonal entry is not positive (context now holds it)");
  ampcg_status ps = refresh_precond(c);
  return ps != AMPCG_OK ? ps : fill_block_layout(c);
}

extern "C" ampcg_status ampcg_adjoint(ampcg_t c, const double* x, const double* dLdx, double tol,
                                      int maxit, const ampcg_policy* policy, double* lambda,
                                      double* dLdA_vals, ampcg_result* res) {
  if (!c || !dLdx || !lambda) return fail(AMPCG_ERR_INVALID_ARG, "NULL argument");
  if (dLdA_vals && !x) return fail(AMPCG_ERR_INVALID_ARG, "x is needed for dL/dA");
  cudaStream_t s = c->stream;
  size_t vb = (size_t)c->n * sizeof(double);
  // lambda starts from zero: A lambda = dL/dx with the same mixed-precision PCG (A = A^T)
  bool l_dev = is_device_ptr(lambda);
  if (l_dev) CUDA_TRY(cudaMemsetAsync(lambda, 0, vb, s));
  else memset(lambda, 0, vb);
  ampcg_status st = solve_impl(c, dLdx, lambda, tol, maxit, policy, res, nullptr);
  if (st != AMPCG_OK && st != AMPCG_NOT_CONVERGED) return st;
  if (!dLdA_vals) return st;
  // the final iterate (lambda) is still in the context's x buffer; x goes to scratch t
  bool x_dev = is_device_ptr(x), g_dev = is_device_ptr(dLdA_vals);
  CUDA_TRY(cudaMemcpyAsync(c->t, x, vb, x_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  double* out = dLdA_vals;
  double* tmp = nullptr;
  if (!g_dev) {
    ampcg_status as = dalloc(&tmp, c->nnz);
    if (as != AMPCG_OK) return as;
    out = tmp;
  }
  Sell A = c->sell();
  if (c->idx16) k_grad_pattern<1><<<c->g_rows, kBlock, 0, s>>>(A, c->rowptr, c->x, c->t, out);
  else k_grad_pattern<0><<<c->g_rows, kBlock, 0, s>>>(A, c->rowptr, c->x, c->t, out);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && tmp)
    e = cudaMemcpyAsync(dLdA_vals, tmp, c->nnz * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return fail(AMPCG_ERR_CUDA, "adjoint gradient: %s", cudaGetErrorString(e));
  return st;
}


// ---------------------------------------------------------------------------
// Log-coefficient field: assembly A(theta) and the chain dL/dtheta.

extern "C" ampcg_status ampcg_assemble_log_coeff(ampcg_t c, const double* theta, const int32_t* nbound) {
  if (!c || !theta || !nbound) return fail(AMPCG_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = c->stream;
  size_t vb = (size_t)c->n * sizeof(double);
  double* d_t = nullptr;
  int* d_nb = nullptr;
  int* flags = nullptr;
  ampcg_status st;
  if ((st = dalloc(&d_t, c->n)) != AMPCG_OK) return st;
  if ((st = dalloc(&d_nb, c->n)) != AMPCG_OK) { cudaFree(d_t); return st; }
  if ((st = dalloc(&flags, 1)) != AMPCG_OK) { cudaFree(d_t); cudaFree(d_nb); return st; }
  cudaError_t e = cudaMemcpyAsync(d_t, theta, vb, is_device_ptr(theta) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_nb, nbound, c->n * sizeof(int), is_device_ptr(nbound) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, sizeof(int), s);
  Sell A = c->sell();
  if (e == cudaSuccess) {
    if (c->idx16) k_assemble_logcoeff<1><<<c->g_rows, kBlock, 0, s>>>(A, d_t, d_nb, c->v64, c->v32, c->dinv64, c->dinv32, c->dinv16, flags);
    else k_assemble_logcoeff<0><<<c->g_rows, kBlock, 0, s>>>(A, d_t, d_nb, c->v64, c->v32, c->dinv64, c->dinv32, c->dinv16, flags);
    e = cudaGetLastError();
  }
  int hf = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_t);
  cudaFree(d_nb);
  cudaFree(flags);
  if (e != cudaSuccess) return fail(AMPCG_ERR_CUDA, "assemble: %s", cudaGetErrorString(e));
  if (hf & 4) return fail(AMPCG_ERR_INVALID_ARG, "a row has no stored diagonal entry");
  ampcg_status ps = refresh_precond(c);
  return ps != AMPCG_OK ? ps : fill_block_layout(c);
}

extern "C" ampcg_status ampcg_grad_log_coeff(ampcg_t c, const double* x, const double* lambda,
                                             double* dLdtheta) {
  if (!c || !x || !lambda || !dLdtheta) return fail(AMPCG_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = c->stream;
  size_t vb = (size_t)c->n * sizeof(double);
  // x -> scratch t, lambda -> scratch r64, result -> b-sized scratch (q buffer)
  CUDA_TRY(cudaMemcpyAsync(c->t, x, vb, is_device_ptr(x) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(c->r64, lambda, vb, is_device_ptr(lambda) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  double* out = (double*)c->q;
  Sell A = c->sell();
  if (c->idx16) k_grad_logcoeff<1><<<c->g_rows, kBlock, 0, s>>>(A, c->t, c->r64, out);
  else k_grad_logcoeff<0><<<c->g_rows, kBlock, 0, s>>>(A, c->t, c->r64, out);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(dLdtheta, out, vb, is_device_ptr(dLdtheta) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return AMPCG_OK;
}


// ---------------------------------------------------------------------------
// Block CSR input: expanded on the device into scalar CSR, then the same
// preparation as ampcg_create_csr.

extern "C" ampcg_status ampcg_create_bsr(ampcg_t* out, int64_t nb, int bs, int64_t nnzb,
                                         const int32_t* browptr, const int32_t* bcolind,
                                         const double* bvals, const ampcg_precond_spec* M,
                                         void* cuda_stream) {
  if (!out) return fail(AMPCG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nb <= 0 || bs < 1 || bs > 16 || nnzb < 0 || !browptr || (nnzb > 0 && (!bcolind || !bvals)))
    return fail(AMPCG_ERR_INVALID_ARG, "need nb > 0, 1 <= bs <= 16, nnzb >= 0 and the three arrays");
  int64_t n = nb * bs, nnz = nnzb * bs * bs;
  if (n > (int64_t)0x7fffffe0 || nnz > (int64_t)0x7fffffff)
    return fail(AMPCG_ERR_INVALID_ARG, "expanded matrix too large for int32 indices");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(AMPCG_ERR_NO_DEVICE, "no CUDA device visible");
  }
  // block row pointer validation on the host side of the copy
  std::vector<int32_t> hb(nb + 1);
  cudaError_t e = cudaMemcpy(hb.data(), browptr, (nb + 1) * sizeof(int32_t),
                             is_device_ptr(browptr) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost);
  if (e != cudaSuccess) return fail(AMPCG_ERR_CUDA, "copy: %s", cudaGetErrorString(e));
  if (hb[0] != 0 || hb[nb] != nnzb) return fail(AMPCG_ERR_INVALID_ARG, "browptr must run from 0 to nnzb");
  for (int64_t i = 0; i < nb; ++i)
    if (hb[i + 1] < hb[i]) return fail(AMPCG_ERR_INVALID_ARG, "browptr must be nondecreasing");
  int *d_bp = nullptr, *d_bc = nullptr, *d_rp = nullptr, *d_c = nullptr;
  double *d_bv = nullptr, *d_v = nullptr;
  ampcg_status st = AMPCG_OK;
  auto cleanup = [&]() {
    cudaFree(d_bp); cudaFree(d_bc); cudaFree(d_rp); cudaFree(d_c); cudaFree(d_bv); cudaFree(d_v);
  };
  if ((st = dalloc(&d_bp, nb + 1)) != AMPCG_OK || (st = dalloc(&d_bc, nnzb)) != AMPCG_OK ||
      (st = dalloc(&d_bv, nnzb * bs * bs)) != AMPCG_OK || (st = dalloc(&d_rp, n + 1)) != AMPCG_OK ||
      (st = dalloc(&d_c, nnz)) != AMPCG_OK || (st = dalloc(&d_v, nnz)) != AMPCG_OK) {
    cleanup();
    return st;
  }
  e = cudaMemcpy(d_bp, hb.data(), (nb + 1) * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && nnzb)
    e = cudaMemcpy(d_bc, bcolind, nnzb * sizeof(int), is_device_ptr(bcolind) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
  if (e == cudaSuccess && nnzb)
    e = cudaMemcpy(d_bv, bvals, nnzb * bs * bs * sizeof(double), is_device_ptr(bvals) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_bsr_expand<<<(int)((n + kBlock - 1) / kBlock), kBlock>>>(nb, bs, d_bp, d_bc, d_bv, d_rp, d_c, d_v);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cleanup();
    return fail(AMPCG_ERR_CUDA, "block expansion: %s", cudaGetErrorString(e));
  }
  st = ampcg_create_csr(out, n, nnz, d_rp, d_c, d_v, M, cuda_stream);
  cleanup();
  if (st != AMPCG_OK) return st;
  // 3 x 3 blocks in rows wider than the staged path's slices (which would keep
  // the scalar layout's uniform-offset slices): the block-row kernels
  if (bs == 3 && (*out)->maxw > kStageW && !(*out)->use_loop) {
    ampcg_layout lay;
    st = ampcg_layout_stats(*out, &lay);
    if (st == AMPCG_OK && lay.stored_uniform == 0) st = build_block_layout(*out);
    if (st != AMPCG_OK) {
      ampcg_destroy(*out);
      *out = nullptr;
    }
  }
  return st;
}


// ---------------------------------------------------------------------------
// Autotuning of the persistent iteration kernel's form.
//
// Per precision pair the kernel can run the four-barrier iteration (the
// scaling and preconditioning in their own step) or, where the scale mode
// allows, the three-barrier one (z_{k+1}, rho_{k+1} formed in the update step
// and reduced with delta_{k+1}).  Which is faster depends on the pair and the
// matrix: the three-barrier form saves a grid barrier but writes and re-reads
// z in u_z (2 bytes a row in binary16, 8 in binary64).  ampcg_tune measures
// both on the context's own matrix and keeps the faster; results are cached
// per matrix shape within the process.

namespace {
struct TuneKey {
  int device;
  int64_t n, nnz, stored;
  int maxw, idx16, mtype, scale;
  bool operator==(const TuneKey& o) const {
    return device == o.device && n == o.n && nnz == o.nnz && stored == o.stored && maxw == o.maxw &&
           idx16 == o.idx16 && mtype == o.mtype && scale == o.scale;
  }
};
std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, ampcg_tuning>> g_tune_cache;

TuneKey tune_key(const ampcg_ctx* c, int scale) {
  return TuneKey{c->device, c->n, c->nnz, c->stored, c->maxw, c->idx16, c->mtype, scale};
}

// Device time of `maxit` iterations of one fixed pair (plus the fixed costs
// of a solve: copies, initial and true residual), CUDA events on the
// context's stream.
ampcg_status time_fixed_pair(ampcg_ctx* c, int ph, int scale, int maxit, const double* b, double* x,
                             float* ms) {
  ampcg_policy pol;
  ampcg_policy_default(&pol);
  pol.criterion = AMPCG_CRIT_FIXED;
  pol.fixed_uz = ph / 2;
  pol.fixed_ur = ph % 2;
  pol.scale = scale;
  pol.verify_refresh = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(AMPCG_ERR_CUDA, "event creation failed");
  }
  ampcg_result res;
  memset(&res, 0, sizeof(res));
  cudaEventRecord(e0, c->stream);
  ampcg_status st = solve_impl(c, b, x, 1e-300, maxit, &pol, &res, nullptr);
  cudaEventRecord(e1, c->stream);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(AMPCG_ERR_CUDA, "tuning events: %s", cudaGetErrorString(e));
  // a pair that breaks down on this system (e.g. binary16 z without scaling)
  // or stops early cannot be timed: AMPCG_NOT_CONVERGED tells the caller
  if (st == AMPCG_ERR_BREAKDOWN || st == AMPCG_ERR_NONFINITE || (st == AMPCG_OK && res.iters != maxit) ||
      (st == AMPCG_NOT_CONVERGED && res.iters != maxit))
    return AMPCG_NOT_CONVERGED;
  if (st != AMPCG_NOT_CONVERGED && st != AMPCG_OK) return st;
  return AMPCG_OK;
}
}  // namespace


extern "C" ampcg_status ampcg_set_tuning(ampcg_t c, int scale, const ampcg_tuning* t) {
  if (!c || !t) return fail(AMPCG_ERR_INVALID_ARG, "NULL argument");
  const int sl = scale_slot(scale);
  if (sl < 0) return fail(AMPCG_ERR_INVALID_ARG, "AMPCG_SCALE_L2 has one form of the iteration kernel");
  for (int ph = 0; ph < 6; ++ph)
    if (t->fused[ph] < -1 || t->fused[ph] > 1) return fail(AMPCG_ERR_INVALID_ARG, "fused[%d] must be -1, 0 or 1", ph);
  for (int ph = 0; ph < 6; ++ph) c->loop_form[sl][ph] = t->fused[ph];
  return AMPCG_OK;
}

extern "C" ampcg_status ampcg_tune(ampcg_t c, int scale, int iters, int pairs, ampcg_tuning* out) {
  if (!c || !out) return fail(AMPCG_ERR_INVALID_ARG, "NULL argument");
  const int sl = scale_slot(scale);
  if (sl < 0) return fail(AMPCG_ERR_INVALID_ARG, "AMPCG_SCALE_L2 has one form of the iteration kernel");
  if (iters < 1 || iters > 10000) return fail(AMPCG_ERR_INVALID_ARG, "iters must be in [1, 10000]");
  if (pairs < 0 || pairs > 63) return fail(AMPCG_ERR_INVALID_ARG, "pairs is a mask of 6 bits");
  if (pairs == 0) pairs = 63;
  memset(out, 0, sizeof(*out));
  for (int ph = 0; ph < 6; ++ph) out->fused[ph] = -1;
  out->iters = iters;
  if (!c->use_loop) return AMPCG_OK;   // no persistent iteration kernel: nothing to choose
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const TuneKey key = tune_key(c, scale);
    for (auto& kv : g_tune_cache) {
      if (kv.first == key && kv.second.iters == iters && (kv.second.reserved & pairs) == pairs) {
        *out = kv.second;
        out->cached = 1;
        for (int ph = 0; ph < 6; ++ph)
          if ((pairs >> ph) & 1) c->loop_form[sl][ph] = out->fused[ph];
        return AMPCG_OK;
      }
    }
  }
  cudaSetDevice(c->device);
  double* b = nullptr;
  double* x = nullptr;
  const size_t vb = (size_t)c->n * sizeof(double);
  ampcg_status st = dalloc(&b, c->n);
  if (st == AMPCG_OK) st = dalloc(&x, c->n);
  std::vector<double> ones((size_t)c->n, 1.0);
  if (st == AMPCG_OK && cudaMemcpy(b, ones.data(), vb, cudaMemcpyHostToDevice) != cudaSuccess)
    st = fail(AMPCG_ERR_CUDA, "tuning right-hand side copy failed");
  int saved[6];
  for (int ph = 0; ph < 6; ++ph) saved[ph] = c->loop_form[sl][ph];
  constexpr int kReps = 3;   // best of kReps timings of each solve length
  for (int ph = 0; ph < 6 && st == AMPCG_OK; ++ph) {
    if (!((pairs >> ph) & 1)) continue;
    double us[2] = {0.0, 0.0}, whole[2] = {0.0, 0.0};
    bool timed = true;
    for (int f = 0; f < 2 && st == AMPCG_OK && timed; ++f) {
      c->loop_form[sl][ph] = f;
      float w = 0.f, t1 = 1e30f, t2 = 1e30f;
      st = time_fixed_pair(c, ph, scale, iters, b, x, &w);   // warm-up (graph build)
      for (int r = 0; r < kReps && st == AMPCG_OK; ++r) {
        float a1 = 0.f, a2 = 0.f;
        st = time_fixed_pair(c, ph, scale, iters, b, x, &a1);
        if (st == AMPCG_OK) st = time_fixed_pair(c, ph, scale, 2 * iters, b, x, &a2);
        t1 = a1 < t1 ? a1 : t1;
        t2 = a2 < t2 ? a2 : t2;
      }
      if (st == AMPCG_NOT_CONVERGED) {   // the pair does not run on this system: not timed
        timed = false;
        st = AMPCG_OK;
      }
      us[f] = 1e3 * (double)(t2 - t1) / iters;
      whole[f] = 1e3 * (double)t2 / (2.0 * iters);
    }
    if (st != AMPCG_OK) break;
    if (!timed) continue;                // fused[ph] stays -1 (automatic)
    // on a small system the fixed costs of a solve can swamp the difference:
    // then both forms are compared on their whole 2 iters solves
    if (!(us[0] > 0.0) || !(us[1] > 0.0)) {
      us[0] = whole[0];
      us[1] = whole[1];
    }
    out->us_plain[ph] = us[0];
    out->us_fused[ph] = us[1];
    out->fused[ph] = us[1] < us[0] ? 1 : 0;
  }
  for (int ph = 0; ph < 6; ++ph) c->loop_form[sl][ph] = saved[ph];
  cudaFree(b);
  cudaFree(x);
  if (st != AMPCG_OK) return st;
  out->reserved = pairs;
  for (int ph = 0; ph < 6; ++ph)
    if ((pairs >> ph) & 1) c->loop_form[sl][ph] = out->fused[ph];
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache.emplace_back(tune_key(c, scale), *out);
  return AMPCG_OK;
}

// ---------------------------------------------------------------------------
// Many independent systems in one call.

// Systems the persistent batched kernel takes (one block per system): at most
// kBatchRows rows, Jacobi or no preconditioner.  Larger systems and Chebyshev
// contexts run as independent device loops on library streams.
constexpr int64_t kBatchRows = 1 << 17;

static bool batch_eligible(const ampcg_ctx* c) {
  return c->n <= kBatchRows && c->mtype != M_CHEBYSHEV;
}

// One persistent launch per column-index width over the eligible systems
// (idx[]), on stream s.  Fills results for them.
static ampcg_status batched_persistent(const std::vector<int>& idx, ampcg_t const* systems,
                                       const double* const* b, double* const* x, double tol, int maxit,
                                       const ampcg_policy& pol, ampcg_result* results, cudaStream_t s,
                                       std::vector<ampcg_status>& sts) {
  const int m = (int)idx.size();
  if (m == 0) return AMPCG_OK;
  auto t0 = std::chrono::steady_clock::now();
  std::vector<BatchSys> hs(m);
  std::vector<char> bdev(m), xdev(m);
  for (int q = 0; q < m; ++q) {
    ampcg_ctx* c = systems[idx[q]];
    ampcg_status hs_ = ensure_hist(c, maxit);
    if (hs_ != AMPCG_OK) return hs_;
    BatchSys& D = hs[q];
    D.A = c->sell();
    D.B = c->bufs();
    D.n = c->n;
    D.mt = c->mtype;
    D.delta_hist = c->dhist;
    D.prec_hist = c->phist;
    D.bbuf = c->b;
    bdev[q] = is_device_ptr(b[idx[q]]);
    xdev[q] = is_device_ptr(x[idx[q]]);
    size_t vb = (size_t)c->n * sizeof(double);
    if (bdev[q]) {
      D.b = b[idx[q]];
    } else {
      CUDA_TRY(cudaMemcpyAsync(c->b, b[idx[q]], vb, cudaMemcpyHostToDevice, s));
      D.b = c->b;
    }
    if (xdev[q]) {
      D.x = x[idx[q]];
    } else {
      CUDA_TRY(cudaMemcpyAsync(c->x, x[idx[q]], vb, cudaMemcpyHostToDevice, s));
      D.x = c->x;
    }
  }
  // one queue per column-index width, longest first
  std::vector<int> ord[2];
  for (int q = 0; q < m; ++q) ord[systems[idx[q]]->idx16 ? 1 : 0].push_back(q);
  for (auto& o : ord)
    std::stable_sort(o.begin(), o.end(), [&](int a, int bq) { return hs[a].n > hs[bq].n; });
  DevState tmpl;
  init_state(&tmpl, &pol, tol, maxit, nullptr);
  // device scratch: systems, orders, two queue counters, template, outcomes
  size_t off_sys = 0, off_ord = off_sys + sizeof(BatchSys) * m;
  size_t off_cnt = (off_ord + sizeof(int) * m + 15) & ~(size_t)15;
  size_t off_tmp = (off_cnt + 2 * sizeof(int) + 15) & ~(size_t)15;
  size_t off_out = (off_tmp + sizeof(DevState) + 15) & ~(size_t)15;
  size_t total = off_out + sizeof(BatchOut) * m;
  std::vector<unsigned char> host(total, 0);
  memcpy(host.data() + off_sys, hs.data(), sizeof(BatchSys) * m);
  int* ho = (int*)(host.data() + off_ord);
  int pos = 0;
  for (auto& o : ord)
    for (int q : o) ho[pos++] = q;
  memcpy(host.data() + off_tmp, &tmpl, sizeof(DevState));
  unsigned char* dev = nullptr;
  CUDA_TRY(cudaMallocAsync((void**)&dev, total, s));
  ampcg_status st = AMPCG_OK;
  std::vector<BatchOut> out(m);
  do {
    cudaError_t e = cudaMemcpyAsync(dev, host.data(), total, cudaMemcpyHostToDevice, s);
    int dev_id = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev_id);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
    const BatchSys* dsys = (const BatchSys*)(dev + off_sys);
    const DevState* dtmp = (const DevState*)(dev + off_tmp);
    BatchOut* dout = (BatchOut*)(dev + off_out);
    const int vr = pol.verify_refresh;
    int first = 0;
    for (int g = 0; g < 2 && e == cudaSuccess; ++g) {
      const int cnt = (int)ord[g].size();
      const int* dord = (const int*)(dev + off_ord) + first;
      int* dcnt = (int*)(dev + off_cnt) + g;
      first += cnt;
      if (cnt == 0) continue;
      const int bs = systems[idx[0]]->batch_block == kBatchBlockSmall ? kBatchBlockSmall : kBatchBlock;
      const void* kern = batched_kernel(g, bs);
      const int smem = bs == kBatchBlockSmall ? (g ? batch_smem_bytes<1, kBatchBlockSmall>()
                                                    : batch_smem_bytes<0, kBatchBlockSmall>())
                                              : (g ? batch_smem_bytes<1>() : batch_smem_bytes<0>());
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) break;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, bs, smem) != cudaSuccess ||
          per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
      }
      const int grid = sms * per_sm < cnt ? sms * per_sm : cnt;
      void* kargs[7] = {&dsys, &dord, const_cast<int*>(&cnt), &dcnt, &dtmp, const_cast<int*>(&vr), &dout};
      e = cudaLaunchKernel(kern, dim3(grid), dim3(bs), kargs, (size_t)smem, s);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out.data(), dev + off_out, sizeof(BatchOut) * m, cudaMemcpyDeviceToHost, s);
    for (int q = 0; q < m && e == cudaSuccess; ++q) {
      ampcg_ctx* c = systems[idx[q]];
      if (!xdev[q])
        e = cudaMemcpyAsync(x[idx[q]], c->x, (size_t)c->n * sizeof(double), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = fail(AMPCG_ERR_CUDA, "batched solve: %s", cudaGetErrorString(e));
  } while (0);
  cudaFreeAsync(dev, s);
  if (st != AMPCG_OK) return st;
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int q = 0; q < m; ++q) {
    const BatchOut& o = out[q];
    sts[idx[q]] = o.status == ST_INTERNAL ? AMPCG_ERR_CUDA : (ampcg_status)o.status;
    ampcg_result* r = results ? &results[idx[q]] : nullptr;
    if (!r) continue;
    ampcg_ctx* c = systems[idx[q]];
    int iters = o.iters;
    if (r->relres_hist)
      CUDA_TRY(cudaMemcpy(r->relres_hist, c->dhist, (iters + 1) * sizeof(double), cudaMemcpyDeviceToHost));
    if (r->prec_hist && iters > 0)
      CUDA_TRY(cudaMemcpy(r->prec_hist, c->phist, iters, cudaMemcpyDeviceToHost));
    if (r->relres_hist)
      for (int i = 0; i <= iters; ++i) r->relres_hist[i] /= o.nb;
    r->iters = iters;
    r->converged = o.status == ST_OK;
    r->refreshes = o.refreshes;
    r->status = o.status == ST_INTERNAL ? AMPCG_ERR_CUDA : o.status;
    r->true_relres = o.true_relres;
    r->updated_relres = o.updated_relres;
    for (int j = 0; j < 3; ++j) r->switch_iter[j] = o.switch_iter[j];
    r->seconds = secs;
    // the persistent launches are reported once, with the first system
    int launches = 0;
    for (auto& o : ord) launches += o.empty() ? 0 : 1;
    r->kernel_launches = q == 0 ? launches : 0;
  }
  return AMPCG_OK;
}

extern "C" ampcg_status ampcg_solve_batched(int nsys, ampcg_t const* systems, const double* const* b,
                                            double* const* x, double tol, int maxit,
                                            const ampcg_policy* policy, ampcg_result* results) {
  if (nsys < 0 || (nsys > 0 && (!systems || !b || !x)))
    return fail(AMPCG_ERR_INVALID_ARG, "bad batched arguments");
  if (nsys == 0) return AMPCG_OK;
  if (!(tol >= 0.0) || maxit < 0) return fail(AMPCG_ERR_INVALID_ARG, "need tol >= 0 and maxit >= 0");
  for (int i = 0; i < nsys; ++i) {
    if (!systems[i] || !b[i] || !x[i]) return fail(AMPCG_ERR_INVALID_ARG, "NULL entry %d", i);
    for (int j = 0; j < i; ++j)
      if (systems[j] == systems[i]) return fail(AMPCG_ERR_INVALID_ARG, "system %d appears twice", i);
  }
  ampcg_policy pol;
  if (policy) pol = *policy;
  else ampcg_policy_default(&pol);
  ampcg_status ps = check_policy(&pol);
  if (ps != AMPCG_OK) return ps;
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<int> small, rest;
  for (int i = 0; i < nsys; ++i) (batch_eligible(systems[i]) ? small : rest).push_back(i);
  const int W = (int)(rest.size() < 16 ? rest.size() : 16);
  const int NS = W + (small.empty() ? 0 : 1);   // stream W: the persistent path
  std::vector<cudaStream_t> ws(NS, nullptr);
  cudaEvent_t ev = nullptr;
  ampcg_status st = AMPCG_OK;
  auto cleanup = [&]() {
    for (cudaStream_t s : ws)
      if (s) cudaStreamDestroy(s);
    if (ev) cudaEventDestroy(ev);
  };
  for (int w = 0; w < NS; ++w) {
    if (cudaStreamCreateWithFlags(&ws[w], cudaStreamNonBlocking) != cudaSuccess) {
      cleanup();
      return fail(AMPCG_ERR_CUDA, "stream creation failed");
    }
  }
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
    cleanup();
    return fail(AMPCG_ERR_CUDA, "event creation failed");
  }
  // work queued on the systems' own streams (their inputs) comes first
  for (int i = 0; i < nsys; ++i) {
    cudaEventRecord(ev, systems[i]->stream);
    for (int w = 0; w < NS; ++w) cudaStreamWaitEvent(ws[w], ev, 0);
  }
  std::vector<ampcg_status> sts(nsys, AMPCG_OK);
  std::vector<std::string> errs(nsys);
  ampcg_status pst = AMPCG_OK;
  std::string perr;
  std::thread pth;
  if (!small.empty()) {
    pth = std::thread([&]() {
      cudaSetDevice(dev);
      pst = batched_persistent(small, systems, b, x, tol, maxit, pol, results, ws[W], sts);
      if (pst != AMPCG_OK) perr = g_err;
    });
  }
  std::atomic<int> next(0);
  auto worker = [&](int w) {
    cudaSetDevice(dev);
    for (;;) {
      int q = next.fetch_add(1);
      if (q >= (int)rest.size()) break;
      int i = rest[q];
      ampcg_result* r = results ? &results[i] : nullptr;
      sts[i] = solve_impl(systems[i], b[i], x[i], tol, maxit, &pol, r, nullptr, ws[w]);
      if (sts[i] != AMPCG_OK && sts[i] != AMPCG_NOT_CONVERGED) errs[i] = g_err;
    }
  };
  std::vector<std::thread> th;
  for (int w = 0; w < W; ++w) th.emplace_back(worker, w);
  for (auto& t : th) t.join();
  if (pth.joinable()) pth.join();
  // later work on the systems' streams waits for the batch
  for (int w = 0; w < NS; ++w) {
    cudaEventRecord(ev, ws[w]);
    for (int i = 0; i < nsys; ++i) cudaStreamWaitEvent(systems[i]->stream, ev, 0);
  }
  cleanup();
  if (pst != AMPCG_OK) {
    g_err = "batched kernel: " + perr;
    return pst;
  }
  for (int i = 0; i < nsys; ++i) {
    if (sts[i] == AMPCG_NOT_CONVERGED && st == AMPCG_OK) st = AMPCG_NOT_CONVERGED;
    if (sts[i] != AMPCG_OK && sts[i] != AMPCG_NOT_CONVERGED) {
      g_err = "system " + std::to_string(i) + ": " + (errs[i].empty() ? ampcg_status_string(sts[i]) : errs[i]);
      return sts[i];
    }
  }
  return st;
}

// ---------------------------------------------------------------------------
// Autotuning of the batched kernel's block size: 1024 threads (one system
// per SM) or 512 (two per SM).  Large systems favour the wide block, many
// small ones the narrow blocks; the batch's own mix decides, by measurement.

extern "C" ampcg_status ampcg_tune_batched(int nsys, ampcg_t const* systems, const ampcg_policy* policy,
                                           int iters, ampcg_batch_tuning* out) {
  if (nsys < 1 || !systems || !out) return fail(AMPCG_ERR_INVALID_ARG, "bad batched tuning arguments");
  if (iters < 1 || iters > 10000) return fail(AMPCG_ERR_INVALID_ARG, "iters must be in [1, 10000]");
  memset(out, 0, sizeof(*out));
  int64_t total = 0;
  for (int i = 0; i < nsys; ++i) {
    if (!systems[i]) return fail(AMPCG_ERR_INVALID_ARG, "NULL system %d", i);
    total += systems[i]->n;
  }
  ampcg_policy pol;
  if (policy) pol = *policy;
  else ampcg_policy_default(&pol);
  ampcg_status st = check_policy(&pol);
  if (st != AMPCG_OK) return st;
  pol.verify_refresh = 0;
  double* b = nullptr;
  double* x = nullptr;
  if ((st = dalloc(&b, total)) != AMPCG_OK) return st;
  if ((st = dalloc(&x, total)) != AMPCG_OK) { cudaFree(b); return st; }
  std::vector<double> ones((size_t)total, 1.0);
  std::vector<const double*> bp((size_t)nsys);
  std::vector<double*> xp((size_t)nsys);
  int64_t off = 0;
  for (int i = 0; i < nsys; ++i) {
    bp[(size_t)i] = b + off;
    xp[(size_t)i] = x + off;
    off += systems[i]->n;
  }
  std::vector<int> saved((size_t)nsys);
  for (int i = 0; i < nsys; ++i) saved[(size_t)i] = systems[i]->batch_block;
  if (cudaMemcpy(b, ones.data(), (size_t)total * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    st = fail(AMPCG_ERR_CUDA, "tuning right-hand sides copy failed");
  const int cand[2] = {kBatchBlock, kBatchBlockSmall};
  for (int j = 0; j < 2 && st == AMPCG_OK; ++j) {
    for (int i = 0; i < nsys; ++i) systems[i]->batch_block = cand[j];
    double best = 0.0;
    for (int rep = 0; rep < 3 && st == AMPCG_OK; ++rep) {   // the first run is a warm-up
      if (cudaMemset(x, 0, (size_t)total * sizeof(double)) != cudaSuccess) {
        st = fail(AMPCG_ERR_CUDA, "tuning memset failed");
        break;
      }
      auto t0 = std::chrono::steady_clock::now();
      st = ampcg_solve_batched(nsys, systems, bp.data(), xp.data(), 1e-300, iters, &pol, nullptr);
      const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      if (st == AMPCG_NOT_CONVERGED) st = AMPCG_OK;
      if (rep == 1 || (rep > 1 && ms < best)) best = ms;
    }
    out->block[j] = cand[j];
    out->ms[j] = best;
  }
  cudaFree(b);
  cudaFree(x);
  const int choice = (st == AMPCG_OK && out->ms[1] < out->ms[0]) ? kBatchBlockSmall : kBatchBlock;
  for (int i = 0; i < nsys; ++i) systems[i]->batch_block = st == AMPCG_OK ? choice : saved[(size_t)i];
  out->chosen = choice;
  out->iters = iters;
  return st;
}

extern "C" ampcg_status ampcg_set_batch_block(int nsys, ampcg_t const* systems, int block) {
  if (nsys < 0 || (nsys > 0 && !systems)) return fail(AMPCG_ERR_INVALID_ARG, "bad arguments");
  if (block != 0 && block != kBatchBlock && block != kBatchBlockSmall)
    return fail(AMPCG_ERR_INVALID_ARG, "block must be 0, %d or %d", kBatchBlock, kBatchBlockSmall);
  for (int i = 0; i < nsys; ++i) {
    if (!systems[i]) return fail(AMPCG_ERR_INVALID_ARG, "NULL system %d", i);
    systems[i]->batch_block = block;
  }
  return AMPCG_OK;
}
