// Allocation-free FP64 solve (gcp_solve_noalloc).
//
// Who needs it: callers that must not allocate device memory at solve time.
// Examples: a host program whose memory pool has already reserved the GPU's
// memory (a cudaMalloc would fail or fragment it), a latency-bound loop that
// cannot afford the implicit device synchronisation of cudaMalloc/cudaFree,
// or code that may not create a library handle.  gcp_solve keeps its
// workspace in a handle that grows with cudaMalloc; this entry point instead
// uses one file-scope __device__ array of fixed size, so it never allocates.
//
// Limits and sharing rules:
//   * M <= kNoAllocMaxM (512): the array holds two FP64 iterates, D^2 and the
//     per-tile partial sums, 6.3 MB in total.  Every GPU that loads the
//     library keeps this array until the process exits.
//   * All calls on a device share the one array, and it keeps the contents
//     of the previous call.  The solver state is cleared at the start of each
//     call; everything else is written before it is read.  Calls whose work
//     overlaps on the GPU (two host threads, or two streams without ordering)
//     race on the array and give wrong results: order them.
//   * The first call on a device looks up the device address of the array
//     (cudaGetSymbolAddress) with that device current and caches it.
//   * The iteration loop is driven from the host: every step ends with a
//     read of the solver state and a stream synchronisation, so the call is
//     synchronous and must not be made while its stream is being captured.
//   * FP64 products only (the arithmetic of gcp_solve with GCP_FP64);
//     GCP_MIXED_AUTO takes that path too.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "gcp_internal.cuh"

using namespace gcp;

namespace {

constexpr int kNoAllocMaxM = 512;
constexpr size_t kMat = (size_t)kNoAllocMaxM * kNoAllocMaxM;
// per-tile partials of the FP64 GEMM1 at the largest size, and the
// per-block partials of the guess and energy reductions
constexpr size_t kPartN = 256 * kPartFields;
constexpr size_t kGpartN = 512;
constexpr size_t kStateN = (sizeof(State) + sizeof(double) - 1) / sizeof(double);
constexpr size_t kScratchDoubles = 3 * kMat + kPartN + kGpartN + kStateN + 32;

// The workspace: D (two ping-pong buffers), S = D^2, partial sums, state.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_base[kMaxDevices] = {nullptr};

void set_err(char* err, int errlen, const char* fmt, ...) {
  if (!err || errlen <= 0) return;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(err, (size_t)errlen, fmt, ap);
  va_end(ap);
}

// Device address of the array on the current device (looked up once).
double* scratch_base(char* err, int errlen, gcp_status* st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_err(err, errlen, "gcp_solve_noalloc: no usable CUDA device (%s)", cudaGetErrorString(e));
    *st = GCP_ERR_CUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_base[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_err(err, errlen, "gcp_solve_noalloc: cudaGetSymbolAddress failed (%s)",
              cudaGetErrorString(e));
      *st = GCP_ERR_CUDA;
      return nullptr;
    }
    g_base[dev] = (double*)p;
  }
  return g_base[dev];
}

}  // namespace

extern "C" gcp_status gcp_solve_noalloc(const void* H, int M, int N, int ld, int h_dtype,
                                        void* D_out, int ldd, int d_dtype, gcp_result* res,
                                        const gcp_options* opt, char* err, int errlen) {
  gcp_options o;
  if (opt)
    o = *opt;
  else
    gcp_default_options(&o);
  if (res) memset(res, 0, sizeof *res);
  if (M > kNoAllocMaxM) {
    set_err(err, errlen, "gcp_solve_noalloc: M = %d exceeds the fixed workspace (M <= %d)", M,
            kNoAllocMaxM);
    return GCP_ERR_INVALID_ARG;
  }
  if (!H || !D_out || M <= 0 || N < 0 || N > M || ld < M || ldd < M ||
      (h_dtype != GCP_F64 && h_dtype != GCP_F32) || (d_dtype != GCP_F64 && d_dtype != GCP_F32) ||
      o.max_iter < 0 || !(o.tol >= 0.0) || (o.stop != 0 && o.stop != 1) ||
      o.guess < GCP_GUESS_CANONICAL || o.guess > GCP_GUESS_HOLE ||
      (o.method != GCP_METHOD_HPCP && o.method != GCP_METHOD_PMCP)) {
    set_err(err, errlen, "gcp_solve_noalloc: bad arguments");
    return GCP_ERR_INVALID_ARG;
  }
  if (o.prec == GCP_MIXED_AUTO) o.prec = GCP_FP64;  // the only arithmetic here
  if (o.prec != GCP_FP64 || o.history_cap != 0) {
    set_err(err, errlen, "gcp_solve_noalloc: only prec = GCP_FP64 without history");
    return GCP_ERR_UNSUPPORTED;
  }
  if ((size_t)f64_num_tiles(M) * kPartFields > kPartN ||
      (size_t)guess_partial_blocks(M) * kGuessFields > kGpartN) {
    set_err(err, errlen, "gcp_solve_noalloc: partial-sum area too small for M = %d", M);
    return GCP_ERR_INVALID_ARG;
  }
  gcp_status rs = GCP_OK;
  double* base = scratch_base(err, errlen, &rs);
  if (!base) return rs;
  double* D0 = base;
  double* D1 = base + kMat;
  double* S = base + 2 * kMat;
  double* part = base + 3 * kMat;
  double* gpart = part + kPartN;
  State* st = (State*)(gpart + kGpartN);
  cudaStream_t s = (cudaStream_t)o.stream;
  const int h64 = h_dtype == GCP_F64, d64 = d_dtype == GCP_F64;

#define NA_CK(call)                                                                         \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      set_err(err, errlen, "gcp_solve_noalloc: %s: %s", #call, cudaGetErrorString(e_));     \
      return GCP_ERR_CUDA;                                                                  \
    }                                                                                       \
  } while (0)

  // the state is the only part that must start at zero
  NA_CK(cudaMemsetAsync(st, 0, sizeof(State), s));
  State hs;
  if (N == 0 || N == M) {
    launch_fill(nullptr, D_out, d64, M, ldd, N == 0 ? 0.0 : 1.0, s);
    launch_energy(D_out, d64, ldd, H, h64, ld, M, gpart, st, s);
    NA_CK(cudaPeekAtLastError());
    NA_CK(cudaMemcpyAsync(&hs, st, sizeof hs, cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    if (res) {
      res->status = GCP_OK;
      res->trace = N;
      res->energy = hs.E;
    }
    return GCP_OK;
  }
  launch_guess_reduce(H, h64, M, ld, gpart, s);
  launch_guess_finalize(gpart, guess_partial_blocks(M), M, N, H, h64, ld, o.guess, st, s);
  launch_state_init(st, 0, s);
  launch_guess_write_d(H, h64, M, ld, D0, 1, M, M, st, s);
  NA_CK(cudaPeekAtLastError());
  Ctl ctl{};
  ctl.M = M;
  ctl.N = N;
  ctl.stop = o.stop;
  ctl.max_iter = o.max_iter;
  ctl.fixed_iters = o.fixed_iters;
  ctl.hist_cap = 0;
  ctl.phase = 0;
  ctl.final_phase = 1;
  ctl.endgame = 0;
  ctl.tol = o.tol;
  ctl.u = kU64;
  ctl.method = o.method;
  double* buf[2] = {D0, D1};
  // The control kernel stops the loop by max_iter (or fixed_iters) steps; the
  // host bound is a guard in 64-bit arithmetic (no overflow for any int
  // option).  A loop that ends without the control kernel's stop reports
  // GCP_ERR_NOT_CONVERGED.
  const long long cap = (long long)(o.fixed_iters > 0 ? o.fixed_iters : o.max_iter) + 2;
  bool stopped = false;
  for (long long it = 0; it < cap; ++it) {
    const int src = (int)(it & 1);
    launch_f64_gemm1(buf[src], S, M, M, nullptr, h64, ld, part, st, s);
    launch_control(part, f64_num_tiles(M), st, nullptr, ctl, 0ull, 0, s);
    launch_f64_gemm2(S, buf[src], buf[src ^ 1], M, M, st, s);
    NA_CK(cudaPeekAtLastError());
    NA_CK(cudaMemcpyAsync(&hs, st, sizeof hs, cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    if (hs.stopped) {
      stopped = true;
      break;
    }
  }
  launch_copy_out_f64(D0, D1, st, M, M, D_out, d64, ldd, s);
  launch_energy(D_out, d64, ldd, H, h64, ld, M, gpart, st, s);
  NA_CK(cudaPeekAtLastError());
  NA_CK(cudaMemcpyAsync(&hs, st, sizeof hs, cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
#undef NA_CK
  if (res) {
    res->status = hs.status;
    res->iters = hs.n;
    res->iters_lowp = 0;
    res->iters_fp64 = hs.n;
    res->trace = hs.T1;
    res->energy = hs.E;
    res->idem_fro = hs.R;
    res->trace_ddbar = hs.T1 - hs.T2;
    res->c_last = hs.c;
    res->mu = hs.mu;
    res->beta2 = hs.beta2;
    res->alpha = hs.alpha;
    res->hmin = hs.hmin;
    res->hmax = hs.hmax;
  }
  if (!stopped && hs.status == GCP_OK) {
    hs.status = GCP_ERR_NOT_CONVERGED;
    if (res) res->status = GCP_ERR_NOT_CONVERGED;
  }
  if (hs.status != GCP_OK)
    set_err(err, errlen, "gcp_solve_noalloc: solve ended: %s", gcp_status_string(hs.status));
  return (gcp_status)hs.status;
}
