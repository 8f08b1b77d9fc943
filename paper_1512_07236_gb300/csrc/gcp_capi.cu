// libgcp C ABI: handle, workspace, graph-captured solve loop and the
// entry points declared in include/gcp.h.
//
// A solve is recorded once into a CUDA graph and replayed while its
// arguments (pointers, sizes, options) stay the same:
//   guess (3 kernels) -> [WHILE split phase: 2 x (GEMM1, control, GEMM2)]
//   -> [transition to FP64] -> [WHILE FP64 phase: 2 x (GEMM1, control, GEMM2)]
//   -> copy-out -> energy.
// The WHILE conditions are set on the device by the control kernel, so the
// host waits only once, for the final scalars.  Each body holds two steps
// because the ping-pong buffers are baked into the captured kernels; a step
// after the stop test fired exits at once.
#include <cuda.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "gcp_internal.cuh"

using namespace gcp;

namespace {

constexpr float kSplitScale = 16384.0f;  // 2^14: see Split in gcp_device.cuh

struct Handle {
  std::string err;
  cudaStream_t cap = nullptr;   // capture stream (solve graphs)
  cudaStream_t body = nullptr;  // capture stream for WHILE bodies
  // FP64 state
  int m64 = 0;
  double* D64[2] = {nullptr, nullptr};
  double* S64 = nullptr;
  // split state (Mp x Mp)
  int mp = 0;
  int tc_bf16 = -1;
  float* X[2] = {nullptr, nullptr};
  void* Xh[2] = {nullptr, nullptr};
  void* Xl[2] = {nullptr, nullptr};
  float* Sig = nullptr;
  void* Sh = nullptr;
  void* Sl = nullptr;
  TcOperands* opX[2] = {nullptr, nullptr};
  TcOperands* opS = nullptr;
  // scratch of the tensor-core kernels (tile hand-over, two slots per CTA)
  float* tcs = nullptr;
  // scalars and partials
  double* part = nullptr;
  size_t part_n = 0;
  double* gpart = nullptr;
  size_t gpart_n = 0;
  State* st = nullptr;
  double* hist = nullptr;
  int hist_cap = 0;
  int hist_last = 0;
  // cached solve graph
  std::vector<char> key;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // batched solves: one arena for every instance's buffers, the instance
  // table, the work lists and a cached graph
  char* arena = nullptr;
  size_t arena_bytes = 0;
  std::vector<char> bkey;
  cudaGraph_t bgraph = nullptr;
  cudaGraphExec_t bexec = nullptr;
  // the batched tensor-core work order chosen by timing: the instance sizes
  // it was chosen for (with the half type), the candidate taken and the
  // GEMM1 times measured (ms; -1 where not timed)
  std::vector<int> tune_key;
  int tune_force = -1;  // gcp_set_batched_order: a fixed candidate, or -1
  int tune_choice = 0;
  double tune_ms[4] = {-1.0, -1.0, -1.0, -1.0};
  // adjoint workspaces (checkpoints, segment iterates, adjoint buffers):
  // FP64 and FP32 (tensor-core) forms
  void* adj = nullptr;
  void* adj_tc = nullptr;
  // exact-slice refinement: nine digit slices of D, row scales, BF16 halves
  // of D and of X = D^2 - D with their tensor maps
  int oz_mp = 0;
  void* oz_slices[kOzSlices] = {nullptr};
  double* oz_rscale = nullptr;
  double* oz_xscale = nullptr;
  void* oz_dh = nullptr;
  void* oz_dl = nullptr;
  void* oz_xh = nullptr;
  void* oz_xl = nullptr;
  OzOperands* oz_op = nullptr;
  TcOperands* oz_opD = nullptr;
  TcOperands* oz_opX = nullptr;
  void* oz_emaps = nullptr;  // device maps of slices 0/1 as split halves (stop test)
};

void free_oz(Handle* h) {
  for (int k = 0; k < kOzSlices; ++k) {
    cudaFree(h->oz_slices[k]);
    h->oz_slices[k] = nullptr;
  }
  cudaFree(h->oz_rscale);
  cudaFree(h->oz_xscale);
  h->oz_xscale = nullptr;
  cudaFree(h->oz_dh);
  cudaFree(h->oz_dl);
  cudaFree(h->oz_xh);
  cudaFree(h->oz_xl);
  h->oz_rscale = nullptr;
  h->oz_dh = h->oz_dl = h->oz_xh = h->oz_xl = nullptr;
  if (h->oz_op) oz_free_operands(h->oz_op);
  if (h->oz_opD) tc_free_operands(h->oz_opD);
  if (h->oz_opX) tc_free_operands(h->oz_opX);
  cudaFree(h->oz_emaps);
  h->oz_emaps = nullptr;
  h->oz_op = nullptr;
  h->oz_opD = h->oz_opX = nullptr;
  h->oz_mp = 0;
}

gcp_status fail(Handle* h, gcp_status s, const char* fmt, ...) {
  if (h) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    h->err = buf;
  }
  return s;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(h, GCP_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));      \
  } while (0)

template <typename T>
cudaError_t grow(T** p, size_t n_old, size_t n_new) {
  if (n_new <= n_old && *p) return cudaSuccess;
  if (*p) cudaFree(*p);
  *p = nullptr;
  return cudaMalloc((void**)p, n_new * sizeof(T));
}

void drop_graph(Handle* h) {
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->exec = nullptr;
  h->graph = nullptr;
  h->key.clear();
}

gcp_status ensure_common(Handle* h, size_t ntiles, int M, int hist_cap) {
  if (!h->st) {
    CK(cudaMalloc((void**)&h->st, sizeof(State)));
    CK(cudaMemset(h->st, 0, sizeof(State)));
  }
  if (ntiles * kPartFields > h->part_n) {
    drop_graph(h);
    CK(grow(&h->part, h->part_n, ntiles * kPartFields));
    h->part_n = ntiles * kPartFields;
  }
  const size_t gp = (size_t)guess_partial_blocks(M) * kGuessFields;
  if (gp > h->gpart_n) {
    drop_graph(h);
    CK(grow(&h->gpart, h->gpart_n, gp));
    h->gpart_n = gp;
  }
  if (hist_cap > h->hist_cap) {
    drop_graph(h);
    CK(grow(&h->hist, (size_t)h->hist_cap * GCP_HISTORY_FIELDS,
            (size_t)hist_cap * GCP_HISTORY_FIELDS));
    h->hist_cap = hist_cap;
  }
  if (!h->cap) CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  if (!h->body) CK(cudaStreamCreateWithFlags(&h->body, cudaStreamNonBlocking));
  return GCP_OK;
}

gcp_status ensure_f64(Handle* h, int M) {
  if (M <= h->m64) return GCP_OK;
  drop_graph(h);
  const size_t n = (size_t)M * M;
  for (int i = 0; i < 2; ++i) {
    if (h->D64[i]) cudaFree(h->D64[i]);
    h->D64[i] = nullptr;
    CK(cudaMalloc((void**)&h->D64[i], n * sizeof(double)));
  }
  if (h->S64) cudaFree(h->S64);
  h->S64 = nullptr;
  CK(cudaMalloc((void**)&h->S64, n * sizeof(double)));
  h->m64 = M;
  return GCP_OK;
}

gcp_status ensure_tcs(Handle* h) {
  if (h->tcs) return GCP_OK;
  drop_graph(h);
  CK(cudaMalloc((void**)&h->tcs, tc_scratch_bytes()));
  return GCP_OK;
}

gcp_status ensure_split(Handle* h, int Mp, int bf16) {
  gcp_status r = ensure_tcs(h);
  if (r != GCP_OK) return r;
  if (Mp == h->mp && bf16 == h->tc_bf16) return GCP_OK;
  drop_graph(h);
  for (int i = 0; i < 2; ++i) {
    if (h->opX[i]) tc_free_operands(h->opX[i]);
    h->opX[i] = nullptr;
  }
  if (h->opS) tc_free_operands(h->opS);
  h->opS = nullptr;
  if (Mp != h->mp) {
    const size_t n = (size_t)Mp * Mp;
    auto fr = [](void* p) {
      if (p) cudaFree(p);
    };
    for (int i = 0; i < 2; ++i) {
      fr(h->X[i]);
      fr(h->Xh[i]);
      fr(h->Xl[i]);
      h->X[i] = nullptr;
      h->Xh[i] = h->Xl[i] = nullptr;
      CK(cudaMalloc((void**)&h->X[i], n * 4));
      CK(cudaMalloc(&h->Xh[i], n * 2));
      CK(cudaMalloc(&h->Xl[i], n * 2));
    }
    fr(h->Sig);
    fr(h->Sh);
    fr(h->Sl);
    h->Sig = nullptr;
    h->Sh = h->Sl = nullptr;
    CK(cudaMalloc((void**)&h->Sig, n * 4));
    CK(cudaMalloc(&h->Sh, n * 2));
    CK(cudaMalloc(&h->Sl, n * 2));
    h->mp = Mp;
  }
  char err[256] = {0};
  for (int i = 0; i < 2; ++i)
    if (tc_make_operands(&h->opX[i], h->Xh[i], h->Xl[i], Mp, bf16, err, sizeof err))
      return fail(h, GCP_ERR_CUDA, "%s", err);
  if (tc_make_operands(&h->opS, h->Sh, h->Sl, Mp, bf16, err, sizeof err))
    return fail(h, GCP_ERR_CUDA, "%s", err);
  h->tc_bf16 = bf16;
  return GCP_OK;
}

gcp_status ensure_oz(Handle* h, int Mp) {
  gcp_status r = ensure_tcs(h);
  if (r != GCP_OK) return r;
  if (Mp == h->oz_mp) return GCP_OK;
  drop_graph(h);
  free_oz(h);
  const size_t n = (size_t)Mp * Mp;
  for (int k = 0; k < kOzSlices; ++k) CK(cudaMalloc(&h->oz_slices[k], n * 2));
  CK(cudaMalloc((void**)&h->oz_rscale, (size_t)Mp * sizeof(double)));
  CK(cudaMalloc((void**)&h->oz_xscale, (size_t)Mp * sizeof(double)));
  CK(cudaMalloc(&h->oz_dh, n * 2));
  CK(cudaMalloc(&h->oz_dl, n * 2));
  CK(cudaMalloc(&h->oz_xh, n * 2));
  CK(cudaMalloc(&h->oz_xl, n * 2));
  char err[256] = {0};
  if (oz_make_operands(&h->oz_op, h->oz_slices, Mp, err, sizeof err) ||
      tc_make_operands(&h->oz_opD, h->oz_dh, h->oz_dl, Mp, 0, err, sizeof err) ||
      tc_make_operands(&h->oz_opX, h->oz_xh, h->oz_xl, Mp, 0, err, sizeof err) ||
      tc_make_device_maps(&h->oz_emaps, h->oz_slices[0], h->oz_slices[1], Mp, err, sizeof err))
    return fail(h, GCP_ERR_CUDA, "%s", err);
  h->oz_mp = Mp;
  return GCP_OK;
}

bool is_split(int prec) { return prec >= GCP_FP16X3 && prec <= GCP_MIXED_BF16; }
bool is_mixed(int prec) { return prec == GCP_MIXED_FP16 || prec == GCP_MIXED_BF16; }
int split_bf16(int prec) { return prec == GCP_BF16X3 || prec == GCP_MIXED_BF16; }

struct SolveArgs {
  const void* H;
  int M, N, ld, h_f64;
  void* D_out;
  int ldd, d_f64;
  gcp_options o;
};

Ctl make_ctl(const SolveArgs& a, int phase, int final_phase) {
  Ctl c{};
  c.endgame = is_split(a.o.prec) ? 1 : 0;
  c.M = a.M;
  c.N = a.N;
  c.stop = a.o.stop;
  c.max_iter = a.o.max_iter;
  c.fixed_iters = a.o.fixed_iters;
  c.hist_cap = a.o.history_cap;
  c.phase = phase;
  c.final_phase = final_phase;
  c.tol = a.o.tol;
  c.u = phase == 1 ? kU32 : kU64;
  c.method = a.o.method;
  return c;
}

// One step of the FP64 phase: GEMM1 -> control -> GEMM2 (buffers src -> dst).
gcp_status rec_f64_step(Handle* h, const SolveArgs& a, int src, Ctl ctl,
                        cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s) {
  const int M = a.M, ld = M;
  const void* Hh = a.o.history_cap > 0 ? a.H : nullptr;
  launch_f64_gemm1(h->D64[src], h->S64, M, ld, Hh, a.h_f64, a.ld, h->part, h->st, s);
  launch_control(h->part, f64_num_tiles(M), h->st, a.o.history_cap > 0 ? h->hist : nullptr, ctl,
                 (unsigned long long)cond, use_cond, s);
  launch_f64_gemm2(h->S64, h->D64[src], h->D64[src ^ 1], M, ld, h->st, s);
  CK(cudaPeekAtLastError());
  return GCP_OK;
}

// One refinement step with exact digit-slice products: slice D -> S = D^2
// (exact) -> traces and ||S - D|| -> control -> D+ = S - 2 (S - D) D - a (S - D)
// (a = 1 - 2c = 0 for the McWeeny step, small when c restores the trace).
gcp_status rec_oz_step(Handle* h, const SolveArgs& a, int src, Ctl ctl,
                       cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s) {
  const int M = a.M, Mp = h->oz_mp;
  launch_oz_slice(h->D64[src], M, Mp, h->oz_slices, h->oz_rscale, h->oz_dh, h->oz_dl, h->st, s);
  if (launch_oz_gemm(h->oz_op, h->oz_rscale, h->S64, M, Mp, oz_weight_cap(M, a.o.tol), h->st, s))
    return fail(h, GCP_ERR_CUDA, "slice GEMM launch failed: %s",
                cudaGetErrorString(cudaGetLastError()));
  launch_oz_finalize(h->S64, h->D64[src], M, Mp, h->part, h->oz_xh, h->oz_xl, h->oz_xscale,
                     h->st, s);
  launch_control(h->part, oz_finalize_blocks(M), h->st, a.o.history_cap > 0 ? h->hist : nullptr,
                 ctl, (unsigned long long)cond, use_cond, s);
  if (tc_launch_mcweeny64(h->oz_opX, h->oz_opD, h->S64, h->D64[src], h->D64[src ^ 1],
                          h->oz_xscale, h->oz_rscale, M, Mp, h->st, h->tcs, s))
    return fail(h, GCP_ERR_CUDA, "McWeeny product launch failed: %s",
                cudaGetErrorString(cudaGetLastError()));
  if (ctl.stop == GCP_STOP_IDEMP_FRO) {
    // stop test of the new iterate D1 from W = D1^2 - D^2 (one split
    // product over [D | Delta | Delta] x [Delta | D | Delta]) instead of a
    // second exact product; the operand buffers of the step are free now
    launch_check_halves(h->D64[src], h->D64[src ^ 1], M, Mp, h->oz_dh, h->oz_dl, h->oz_xh,
                        h->oz_xl, h->oz_slices[0], h->oz_slices[1], h->st, s);
    if (tc_launch_check(h->oz_opD, h->oz_opX, h->oz_emaps, h->S64, h->D64[src ^ 1], h->part, M,
                        Mp, h->st, h->tcs, s))
      return fail(h, GCP_ERR_CUDA, "stop-test product launch failed: %s",
                  cudaGetErrorString(cudaGetLastError()));
    launch_check_control(h->part, tc_num_tiles(Mp), h->st,
                         a.o.history_cap > 0 ? h->hist : nullptr, ctl, (unsigned long long)cond,
                         use_cond, s);
  }
  CK(cudaPeekAtLastError());
  return GCP_OK;
}

bool use_oz(const SolveArgs& a) {
  return is_mixed(a.o.prec) && a.o.refine == 0 && a.o.fixed_iters == 0 && a.M <= 29000;
}

// One step of the split phase on the shifted state.
gcp_status rec_split_step(Handle* h, const SolveArgs& a, int src, Ctl ctl,
                          cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s) {
  const int M = a.M, Mp = h->mp, bf = h->tc_bf16;
  const void* Hh = a.o.history_cap > 0 ? a.H : nullptr;
  if (tc_launch_gemm1(h->opX[src], h->X[src], h->Sig, h->Sh, h->Sl, M, Mp, Hh, a.h_f64, a.ld,
                      h->part, h->st, bf, kSplitScale, h->tcs, s))
    return fail(h, GCP_ERR_CUDA, "tcgen05 GEMM1 launch failed: %s",
                cudaGetErrorString(cudaGetLastError()));
  launch_control(h->part, tc_num_tiles(Mp), h->st, a.o.history_cap > 0 ? h->hist : nullptr, ctl,
                 (unsigned long long)cond, use_cond, s);
  if (tc_launch_gemm2(h->opS, h->opX[src], h->X[src], h->Sig, h->X[src ^ 1], h->Xh[src ^ 1],
                      h->Xl[src ^ 1], M, Mp, h->st, bf, kSplitScale, h->tcs, s))
    return fail(h, GCP_ERR_CUDA, "tcgen05 GEMM2 launch failed: %s",
                cudaGetErrorString(cudaGetLastError()));
  CK(cudaPeekAtLastError());
  return GCP_OK;
}

// Add a WHILE node at the current capture position of `s` and capture its
// body (two steps) on h->body.
template <typename StepFn>
gcp_status rec_while(Handle* h, cudaStream_t s, StepFn step) {
  cudaStreamCaptureStatus cst;
  unsigned long long id = 0;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edata = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(s, &cst, &id, &g, &deps, &edata, &nd));
  cudaGraphConditionalHandle cond;
  CK(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
  p.conditional.handle = cond;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, deps, edata, nd, &p));
  cudaGraph_t bodyg = p.conditional.phGraph_out[0];
  CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  CK(cudaStreamBeginCaptureToGraph(h->body, bodyg, nullptr, nullptr, 0,
                                   cudaStreamCaptureModeRelaxed));
  gcp_status r = step(0, cond, h->body);
  if (r == GCP_OK) r = step(1, cond, h->body);
  cudaGraph_t out = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->body, &out);
  if (r != GCP_OK) return r;
  if (e != cudaSuccess) return fail(h, GCP_ERR_CUDA, "body capture: %s", cudaGetErrorString(e));
  return GCP_OK;
}

// Record the whole solve on stream s (captured, or eager with a host loop).
gcp_status record_solve(Handle* h, const SolveArgs& a, cudaStream_t s, bool graph) {
  const int M = a.M, N = a.N;
  const bool split = is_split(a.o.prec), mixed = is_mixed(a.o.prec);
  launch_guess_reduce(a.H, a.h_f64, M, a.ld, h->gpart, s);
  launch_guess_finalize(h->gpart, guess_partial_blocks(M), M, N, a.H, a.h_f64, a.ld, a.o.guess,
                        h->st, s);
  launch_state_init(h->st, split ? 1 : 0, s);
  if (split) {
    launch_guess_write_x(a.H, a.h_f64, M, a.ld, h->X[0], h->Xh[0], h->Xl[0], h->mp, h->tc_bf16,
                         kSplitScale, h->st, s);
  } else {
    launch_guess_write_d(a.H, a.h_f64, M, a.ld, h->D64[0], 1, M, M, h->st, s);
  }
  CK(cudaPeekAtLastError());
  if (split) {
    const Ctl ctl = make_ctl(a, 1, mixed ? 0 : 1);
    auto step = [&](int src, cudaGraphConditionalHandle c, cudaStream_t ss) {
      return rec_split_step(h, a, src, ctl, c, graph ? 1 : 0, ss);
    };
    if (graph) {
      gcp_status r = rec_while(h, s, step);
      if (r != GCP_OK) return r;
    } else {
      for (int it = 0;; ++it) {
        gcp_status r = step(it & 1, 0, s);
        if (r != GCP_OK) return r;
        State hs;
        CK(cudaMemcpyAsync(&hs, h->st, sizeof hs, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (hs.stopped) break;
      }
    }
  }
  if (mixed) {
    // convert the split iterate (buffer chosen by the parity) before the
    // FP64 phase resets the parity to its own buffer 0
    launch_x_to_d64(h->X[0], h->X[1], h->st, M, h->mp, h->D64[0], M, s);
    launch_phase_begin(h->st, 0, s);
  }
  if (!split || mixed) {
    Ctl ctl = make_ctl(a, 0, 1);
    const bool oz = use_oz(a);
    ctl.mcw_only = oz ? 1 : 0;
    // the slice product's dropped digit pairs (see oz_weight_cap)
    if (oz && ctl.stop == GCP_STOP_IDEMP_FRO) ctl.tol -= oz_tail_estimate(M, a.o.tol);
    ctl.phase_max = mixed ? a.o.refine_iters : 0;
    auto step = [&](int src, cudaGraphConditionalHandle c, cudaStream_t ss) {
      return oz ? rec_oz_step(h, a, src, ctl, c, graph ? 1 : 0, ss)
                : rec_f64_step(h, a, src, ctl, c, graph ? 1 : 0, ss);
    };
    if (graph) {
      gcp_status r = rec_while(h, s, step);
      if (r != GCP_OK) return r;
    } else {
      for (int it = 0;; ++it) {
        gcp_status r = step(it & 1, 0, s);
        if (r != GCP_OK) return r;
        State hs;
        CK(cudaMemcpyAsync(&hs, h->st, sizeof hs, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (hs.stopped) break;
      }
    }
  }
  if (split && !mixed)
    launch_copy_out_x(h->X[0], h->X[1], h->st, M, h->mp, a.D_out, a.d_f64, a.ldd, s);
  else
    launch_copy_out_f64(h->D64[0], h->D64[1], h->st, M, M, a.D_out, a.d_f64, a.ldd, s);
  launch_energy(a.D_out, a.d_f64, a.ldd, a.H, a.h_f64, a.ld, M, h->gpart, h->st, s);
  CK(cudaPeekAtLastError());
  return GCP_OK;
}

std::vector<char> make_key(const SolveArgs& a) {
  std::vector<char> k(sizeof(SolveArgs));
  SolveArgs c = a;
  c.o.stream = nullptr;
  memcpy(k.data(), &c, sizeof c);
  return k;
}

void fill_result(const State& hs, gcp_result* res) {
  if (!res) return;
  res->status = hs.status;
  res->iters = hs.n;
  res->iters_lowp = hs.n_lowp;
  res->iters_fp64 = hs.n - hs.n_lowp;
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

bool valid_dtype(int d) { return d == GCP_F64 || d == GCP_F32; }

bool valid_modes(const gcp_options& o) {
  return o.guess >= GCP_GUESS_CANONICAL && o.guess <= GCP_GUESS_HOLE &&
         (o.method == GCP_METHOD_HPCP || o.method == GCP_METHOD_PMCP) && o.refine_iters >= 0 &&
         (o.check_symmetry == 0 || o.check_symmetry == 1) && o.sym_tol >= 0.0 &&
         o.sym_tol <= 1.0;
}

// GCP_MIXED_AUTO: the FP64 path for small M (the tensor-core tiles would be
// mostly padding and the FP64 products are cheap) or a tolerance below the
// exact-slice refinement's floor, the split-FP16 path with refinement
// otherwise.
constexpr int kAutoMixedMinM = 512;
int resolve_prec(int prec, int M, double tol) {
  if (prec == GCP_FP32) return GCP_FP16X3;  // the same arithmetic for a solve
  if (prec != GCP_MIXED_AUTO) return prec;
  return (M < kAutoMixedMinM || tol < 1e-10) ? GCP_FP64 : GCP_MIXED_FP16;
}

// Optional check that H is symmetric (gcp_options.check_symmetry).
gcp_status check_symmetry(Handle* h, const void* H, int h_f64, int M, int ld, double rel,
                          cudaStream_t s, const char* who) {
  gcp_status r = ensure_common(h, 1, M, 0);
  if (r != GCP_OK) return r;
  launch_sym_check(H, h_f64, M, ld, h->gpart, s);
  double v[2] = {0.0, 0.0};
  CK(cudaMemcpyAsync(v, h->gpart, sizeof v, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (!(v[0] <= rel * v[1]))
    return fail(h, GCP_ERR_INVALID_ARG, "%s: H is not symmetric: max|H_ij - H_ji| = %.3e > %.3e",
                who, v[0], rel * v[1]);
  return GCP_OK;
}

}  // namespace

extern "C" {

void gcp_default_options(gcp_options* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->prec = GCP_FP64;
  o->stop = GCP_STOP_IDEMP_FRO;
  o->tol = 1e-12;
  o->max_iter = 100;
  o->fixed_iters = 0;
  o->ckpt_every = 8;
  o->history_cap = 0;
  o->use_graph = 1;
  o->stream = nullptr;
  o->refine_iters = 0;
  o->check_symmetry = 0;
  o->sym_tol = 0.0;
}

const char* gcp_status_string(int s) {
  switch (s) {
    case GCP_OK: return "ok";
    case GCP_ERR_INVALID_ARG: return "invalid argument";
    case GCP_ERR_NOT_CONVERGED: return "not converged";
    case GCP_ERR_ILL_CONDITIONED: return "ill-conditioned initial guess";
    case GCP_ERR_NO_GAP: return "no gap (H = mu I)";
    case GCP_ERR_NONFINITE: return "non-finite trace";
    case GCP_ERR_TIMEOUT: return "device wait timed out";
    case GCP_ERR_CUDA: return "CUDA error";
    case GCP_ERR_UNSUPPORTED: return "unsupported";
    case GCP_ERR_NO_CHECKPOINT: return "no checkpoint";
    default: return "unknown status";
  }
}

gcp_status gcp_create(void** out) {
  if (!out) return GCP_ERR_INVALID_ARG;
  *out = new Handle;
  return GCP_OK;
}

gcp_status gcp_destroy(void* hv) {
  Handle* h = (Handle*)hv;
  if (!h) return GCP_ERR_INVALID_ARG;
  drop_graph(h);
  if (h->bexec) cudaGraphExecDestroy(h->bexec);
  if (h->bgraph) cudaGraphDestroy(h->bgraph);
  cudaFree(h->arena);
  cudaFree(h->tcs);
  adjoint_free(h->adj);
  adjoint_tc_free(h->adj_tc);
  free_oz(h);
  for (int i = 0; i < 2; ++i) {
    cudaFree(h->D64[i]);
    cudaFree(h->X[i]);
    cudaFree(h->Xh[i]);
    cudaFree(h->Xl[i]);
    if (h->opX[i]) tc_free_operands(h->opX[i]);
  }
  if (h->opS) tc_free_operands(h->opS);
  cudaFree(h->S64);
  cudaFree(h->Sig);
  cudaFree(h->Sh);
  cudaFree(h->Sl);
  cudaFree(h->part);
  cudaFree(h->gpart);
  cudaFree(h->st);
  cudaFree(h->hist);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->body) cudaStreamDestroy(h->body);
  delete h;
  return GCP_OK;
}

const char* gcp_last_error(void* hv) {
  Handle* h = (Handle*)hv;
  return h ? h->err.c_str() : "null handle";
}

gcp_status gcp_init_guess(void* hv, const void* H, int M, int N, int ld, int h_dtype, void* D0,
                          int ldd, int d_dtype, double* info, const gcp_options* opt) {
  Handle* h = (Handle*)hv;
  if (!h) return GCP_ERR_INVALID_ARG;
  if (!H || !D0 || M <= 0 || N <= 0 || N >= M || ld < M || ldd < M || !valid_dtype(h_dtype) ||
      !valid_dtype(d_dtype))
    return fail(h, GCP_ERR_INVALID_ARG, "gcp_init_guess: bad arguments");
  gcp_options o;
  if (opt)
    o = *opt;
  else
    gcp_default_options(&o);
  if (!valid_modes(o)) return fail(h, GCP_ERR_INVALID_ARG, "gcp_init_guess: bad guess or method");
  cudaStream_t s = (cudaStream_t)o.stream;
  gcp_status r = ensure_common(h, 1, M, 0);
  if (r != GCP_OK) return r;
  launch_guess_reduce(H, h_dtype == GCP_F64, M, ld, h->gpart, s);
  launch_guess_finalize(h->gpart, guess_partial_blocks(M), M, N, H, h_dtype == GCP_F64, ld,
                        o.guess, h->st, s);
  launch_guess_write_d(H, h_dtype == GCP_F64, M, ld, D0, d_dtype == GCP_F64, ldd, M, h->st, s);
  CK(cudaPeekAtLastError());
  State hs;
  CK(cudaMemcpyAsync(&hs, h->st, sizeof hs, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (info) {
    info[0] = hs.mu;
    info[1] = hs.beta2;
    info[2] = hs.hmin;
    info[3] = hs.hmax;
    info[4] = hs.theta;
  }
  return hs.no_gap ? fail(h, GCP_ERR_NO_GAP, "H has a zero-width spectrum bound") : GCP_OK;
}

gcp_status gcp_step(void* hv, void* D, int M, int N, int ld, int d_dtype, double* out,
                    const gcp_options* opt) {
  Handle* h = (Handle*)hv;
  if (!h) return GCP_ERR_INVALID_ARG;
  gcp_options o;
  if (opt)
    o = *opt;
  else
    gcp_default_options(&o);
  if (!D || M <= 0 || N < 0 || N > M || ld < M || !valid_dtype(d_dtype) || o.prec < 0 ||
      o.prec > GCP_MIXED_BF16 || !valid_modes(o))
    return fail(h, GCP_ERR_INVALID_ARG, "gcp_step: bad arguments");
  cudaStream_t s = (cudaStream_t)o.stream;
  SolveArgs a{};
  a.H = nullptr;
  a.M = M;
  a.N = N;
  a.ld = ld;
  a.h_f64 = 1;
  a.o = o;
  a.o.fixed_iters = 1;  // one step, no stop test
  a.o.history_cap = 0;
  const bool split = is_split(o.prec) && !is_mixed(o.prec);
  gcp_status r;
  if (split) {
    const int Mp = tc_pad(M);
    if ((r = ensure_common(h, tc_num_tiles(Mp), M, 0)) != GCP_OK) return r;
    if ((r = ensure_split(h, Mp, split_bf16(o.prec))) != GCP_OK) return r;
  } else {
    if ((r = ensure_common(h, f64_num_tiles(M), M, 0)) != GCP_OK) return r;
    if ((r = ensure_f64(h, M)) != GCP_OK) return r;
  }
  // state: theta for the shift, loop fields reset
  State init;
  memset(&init, 0, sizeof init);
  init.theta = (double)N / (double)M;
  CK(cudaMemcpyAsync(h->st, &init, sizeof init, cudaMemcpyHostToDevice, s));
  launch_state_init(h->st, split ? 1 : 0, s);
  if (split) {
    launch_d_to_x(D, d_dtype == GCP_F64, M, ld, h->X[0], h->Xh[0], h->Xl[0], h->mp, h->tc_bf16,
                  kSplitScale, init.theta, s);
    if ((r = rec_split_step(h, a, 0, make_ctl(a, 1, 1), 0, 0, s)) != GCP_OK) return r;
    launch_copy_out_x(h->X[0], h->X[1], h->st, M, h->mp, D, d_dtype == GCP_F64, ld, s);
  } else {
    launch_convert(D, d_dtype == GCP_F64, ld, h->D64[0], 1, M, M, s);
    if ((r = rec_f64_step(h, a, 0, make_ctl(a, 0, 1), 0, 0, s)) != GCP_OK) return r;
    launch_copy_out_f64(h->D64[0], h->D64[1], h->st, M, M, D, d_dtype == GCP_F64, ld, s);
  }
  CK(cudaPeekAtLastError());
  State hs;
  CK(cudaMemcpyAsync(&hs, h->st, sizeof hs, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hs.timeout) return fail(h, GCP_ERR_TIMEOUT, "a device-side wait gave up");
  if (out) {
    out[0] = hs.T1;
    out[1] = hs.T2;
    out[2] = hs.T3;
    out[3] = hs.R;
    out[4] = hs.c;
    out[5] = hs.n > 0 && hs.apply ? 1.0 : 0.0;
  }
  return GCP_OK;
}

gcp_status gcp_solve(void* hv, const void* H, int M, int N, int ld, int h_dtype, void* D_out,
                     int ldd, int d_dtype, gcp_result* res, const gcp_options* opt) {
  Handle* h = (Handle*)hv;
  if (!h) return GCP_ERR_INVALID_ARG;
  gcp_options o;
  if (opt)
    o = *opt;
  else
    gcp_default_options(&o);
  if (!H || !D_out || M <= 0 || N < 0 || N > M || ld < M || ldd < M || !valid_dtype(h_dtype) ||
      !valid_dtype(d_dtype) || o.prec < 0 || o.prec > GCP_FP32 || o.max_iter < 0 ||
      o.history_cap < 0 || !(o.tol >= 0.0) || (o.stop != 0 && o.stop != 1) || !valid_modes(o))
    return fail(h, GCP_ERR_INVALID_ARG, "gcp_solve: bad arguments");
  o.prec = resolve_prec(o.prec, M, o.tol);
  cudaStream_t s = (cudaStream_t)o.stream;
  if (o.check_symmetry) {
    gcp_status r = check_symmetry(h, H, h_dtype == GCP_F64, M, ld, o.sym_tol, s, "gcp_solve");
    if (r != GCP_OK) return r;
  }
  if (res) memset(res, 0, sizeof *res);
  if (N == 0 || N == M) {
    launch_fill(nullptr, D_out, d_dtype == GCP_F64, M, ldd, N == 0 ? 0.0 : 1.0, s);
    CK(cudaPeekAtLastError());
    CK(cudaStreamSynchronize(s));
    if (res) {
      res->status = GCP_OK;
      res->trace = N;
      res->energy = 0.0;
    }
    if (N == M && res) {
      // E = Tr H for D = I: computed by the energy kernel on the filled D
      gcp_status r = ensure_common(h, 1, M, 0);
      if (r != GCP_OK) return r;
      launch_energy(D_out, d_dtype == GCP_F64, ldd, H, h_dtype == GCP_F64, ld, M, h->gpart, h->st,
                    s);
      State hs;
      CK(cudaMemcpyAsync(&hs, h->st, sizeof hs, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      res->energy = hs.E;
    }
    return GCP_OK;
  }
  SolveArgs a{};
  a.H = H;
  a.M = M;
  a.N = N;
  a.ld = ld;
  a.h_f64 = h_dtype == GCP_F64;
  a.D_out = D_out;
  a.ldd = ldd;
  a.d_f64 = d_dtype == GCP_F64;
  a.o = o;
  const bool split = is_split(o.prec), mixed = is_mixed(o.prec);
  gcp_status r;
  size_t nt = 1;
  if (split) nt = tc_num_tiles(tc_pad(M));
  if (!split || mixed) nt = nt > (size_t)f64_num_tiles(M) ? nt : (size_t)f64_num_tiles(M);
  if (use_oz(a)) nt = nt > (size_t)oz_finalize_blocks(M) ? nt : (size_t)oz_finalize_blocks(M);
  if ((r = ensure_common(h, nt, M, o.history_cap)) != GCP_OK) return r;
  if (split && (r = ensure_split(h, tc_pad(M), split_bf16(o.prec))) != GCP_OK) return r;
  if ((!split || mixed) && (r = ensure_f64(h, M)) != GCP_OK) return r;
  if (use_oz(a) && (r = ensure_oz(h, tc_pad(M))) != GCP_OK) return r;
  if (o.use_graph) {
    std::vector<char> key = make_key(a);
    if (!h->exec || key != h->key) {
      drop_graph(h);
      CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeRelaxed));
      r = record_solve(h, a, h->cap, true);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(h->cap, &g);
      if (r != GCP_OK) {
        if (g) cudaGraphDestroy(g);
        return r;
      }
      if (e != cudaSuccess)
        return fail(h, GCP_ERR_CUDA, "solve capture: %s", cudaGetErrorString(e));
      h->graph = g;
      CK(cudaGraphInstantiate(&h->exec, g, 0));
      h->key = key;
    }
    CK(cudaGraphLaunch(h->exec, s));
  } else {
    if ((r = record_solve(h, a, s, false)) != GCP_OK) return r;
  }
  State hs;
  CK(cudaMemcpyAsync(&hs, h->st, sizeof hs, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  h->hist_last = hs.hist_n;
  fill_result(hs, res);
  if (res) res->energy = hs.E;
  if (hs.timeout) return fail(h, GCP_ERR_TIMEOUT, "a device-side wait gave up");
  if (hs.status != GCP_OK)
    return fail(h, (gcp_status)hs.status, "solve ended: %s", gcp_status_string(hs.status));
  return GCP_OK;
}

gcp_status gcp_get_history(void* hv, double* out, int cap, int* n_out) {
  Handle* h = (Handle*)hv;
  if (!h || !out || cap < 0) return GCP_ERR_INVALID_ARG;
  int n = h->hist_last < cap ? h->hist_last : cap;
  if (n > h->hist_cap) n = h->hist_cap;
  if (n > 0) CK(cudaMemcpy(out, h->hist, (size_t)n * GCP_HISTORY_FIELDS * sizeof(double),
                           cudaMemcpyDeviceToHost));
  if (n_out) *n_out = n;
  return GCP_OK;
}

gcp_status gcp_solve_batched(void* hv, int batch, const void* const* H, const int* M, const int* N,
                             const int* ld, int h_dtype, void* const* D_out, int d_dtype,
                             gcp_result* res, const gcp_options* opt) {
  Handle* h = (Handle*)hv;
  if (!h) return GCP_ERR_INVALID_ARG;
  gcp_options o;
  if (opt)
    o = *opt;
  else
    gcp_default_options(&o);
  if (batch <= 0 || !H || !M || !N || !ld || !D_out || !valid_dtype(h_dtype) ||
      !valid_dtype(d_dtype) || o.prec < 0 || o.prec > GCP_FP32 || o.max_iter < 0 ||
      !(o.tol >= 0.0) || (o.stop != 0 && o.stop != 1) || o.history_cap != 0)
    return fail(h, GCP_ERR_INVALID_ARG, "gcp_solve_batched: bad arguments");
  if (!valid_modes(o)) return fail(h, GCP_ERR_INVALID_ARG, "gcp_solve_batched: bad guess or method");
  int maxM_all = 0;
  for (int b = 0; b < batch; ++b) {
    if (!H[b] || !D_out[b] || M[b] <= 0 || N[b] < 0 || N[b] > M[b] || ld[b] < M[b])
      return fail(h, GCP_ERR_INVALID_ARG, "gcp_solve_batched: bad instance %d", b);
    if (M[b] > maxM_all) maxM_all = M[b];
  }
  // one arithmetic for the whole batch, chosen from its largest instance
  o.prec = resolve_prec(o.prec, maxM_all, o.tol);
  cudaStream_t s = (cudaStream_t)o.stream;
  if (o.check_symmetry)
    for (int b = 0; b < batch; ++b) {
      gcp_status r = check_symmetry(h, H[b], h_dtype == GCP_F64, M[b], ld[b], o.sym_tol, s,
                                    "gcp_solve_batched");
      if (r != GCP_OK) return fail(h, r, "%s (instance %d)", h->err.c_str(), b);
    }
  const bool split = is_split(o.prec), mixed = is_mixed(o.prec);
  const int bf16 = split_bf16(o.prec);
  const int h64 = h_dtype == GCP_F64, d64 = d_dtype == GCP_F64;
  if (res) memset(res, 0, sizeof(gcp_result) * (size_t)batch);

  // trivial fillings: D = 0 or D = I, one instance at a time
  std::vector<int> idx;
  gcp_status r = ensure_common(h, 1, 1024, 0);
  if (r != GCP_OK) return r;
  for (int b = 0; b < batch; ++b) {
    if (N[b] == 0 || N[b] == M[b]) {
      if ((r = ensure_common(h, 1, M[b], 0)) != GCP_OK) return r;
      launch_fill(nullptr, D_out[b], d64, M[b], M[b], N[b] == 0 ? 0.0 : 1.0, s);
      launch_energy(D_out[b], d64, M[b], H[b], h64, ld[b], M[b], h->gpart, h->st, s);
      State hs;
      CK(cudaMemcpyAsync(&hs, h->st, sizeof hs, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (res) {
        res[b].status = GCP_OK;
        res[b].trace = N[b];
        res[b].energy = hs.E;
      }
    } else {
      idx.push_back(b);
    }
  }
  const int nb = (int)idx.size();
  if (nb == 0) return GCP_OK;
  if (split && (r = ensure_tcs(h)) != GCP_OK) return r;

  // ---- layout of the arena -------------------------------------------
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  std::vector<BatchItem> items(nb);
  std::vector<size_t> inst_off(nb);
  size_t off = al(sizeof(State) * (size_t)nb);  // states first, contiguous
  int ntc = 0, nf64 = 0, noz = 0, maxM = 0;
  for (int k = 0; k < nb; ++k) maxM = M[idx[k]] > maxM ? M[idx[k]] : maxM;
  // the refinement of the mixed modes: exact digit slices as in gcp_solve
  const bool oz = mixed && o.refine == 0 && o.fixed_iters == 0 && maxM <= 29000;
  for (int k = 0; k < nb; ++k) {
    const int b = idx[k];
    BatchItem& it = items[k];
    memset(&it, 0, sizeof it);
    it.M = M[b];
    it.Mp = tc_pad(M[b]);
    it.N = N[b];
    it.ld = ld[b];
    it.ldd = M[b];
    it.H = H[b];
    it.D_out = D_out[b];
    it.gblocks = guess_partial_blocks(M[b]);
    maxM = M[b] > maxM ? M[b] : maxM;
    inst_off[k] = off;
    if (split) {
      const size_t n2 = (size_t)it.Mp * it.Mp;
      off += al(tc_map_bytes());
      off += 3 * al(n2 * 4) + 6 * al(n2 * 2);
      it.tc_off = ntc;
      it.tc_n = tc_num_tiles(it.Mp);
      ntc += it.tc_n;
    }
    if (!split || mixed) {
      off += 3 * al((size_t)it.M * it.M * 8);
      it.f64_off = nf64;
      it.f64_n = batch_f64_tiles(it.M);
      nf64 += it.f64_n;
    }
    if (oz) {
      const size_t n2 = (size_t)it.Mp * it.Mp;
      off += al(oz_batch_map_bytes()) + (kOzSlices + 4) * al(n2 * 2) +
             2 * al((size_t)it.Mp * 8);
      it.oz_off = noz;
      noz += oz_finalize_blocks(it.M);
    }
  }
  const int nslots = ntc > nf64 ? (ntc > noz ? ntc : noz) : (nf64 > noz ? nf64 : noz);
  const size_t items_off = off;
  off += al(sizeof(BatchItem) * (size_t)nb);
  const size_t tinst_tc_off = off;
  off += al(sizeof(int) * (size_t)(ntc > 0 ? ntc : 1));
  const size_t tinst_f64_off = off;
  off += al(sizeof(int) * (size_t)(nf64 > 0 ? nf64 : 1));
  const size_t order_off = off;
  off += al(sizeof(int) * (size_t)(ntc > 0 ? ntc : 1));
  const size_t part_off = off;
  off += al(sizeof(double) * kPartFields * (size_t)nslots);
  const size_t gpart_off = off;
  const int gstride = guess_partial_blocks(maxM);
  off += al(sizeof(double) * kGuessFields * (size_t)gstride * (size_t)nb);
  const size_t active_off = off;
  off += al(sizeof(int));
  if (off > h->arena_bytes) {
    if (h->bexec) cudaGraphExecDestroy(h->bexec);
    if (h->bgraph) cudaGraphDestroy(h->bgraph);
    h->bexec = nullptr;
    h->bgraph = nullptr;
    h->bkey.clear();
    cudaFree(h->arena);
    h->arena = nullptr;
    h->arena_bytes = 0;
    CK(cudaMalloc((void**)&h->arena, off));
    h->arena_bytes = off;
  }
  char* A = h->arena;
  State* states = (State*)A;
  BatchItem* items_d = (BatchItem*)(A + items_off);
  int* tinst_tc = (int*)(A + tinst_tc_off);
  int* tinst_f64 = (int*)(A + tinst_f64_off);
  int* order_d = (int*)(A + order_off);
  double* part = (double*)(A + part_off);
  double* gpart = (double*)(A + gpart_off);
  int* active = (int*)(A + active_off);

  // key: everything the recorded graph depends on
  std::vector<char> key;
  auto put = [&key](const void* p, size_t n) {
    key.insert(key.end(), (const char*)p, (const char*)p + n);
  };
  {
    gcp_options k = o;
    k.stream = nullptr;
    put(&k, sizeof k);
    put(&batch, sizeof batch);
    put(&h_dtype, sizeof h_dtype);
    put(&d_dtype, sizeof d_dtype);
    put(H, sizeof(void*) * batch);
    put(D_out, sizeof(void*) * batch);
    put(M, sizeof(int) * batch);
    put(N, sizeof(int) * batch);
    put(ld, sizeof(int) * batch);
    put(&h->arena, sizeof h->arena);
  }
  const bool fresh = !(o.use_graph && h->bexec && key == h->bkey);
  if (fresh) {
    // fill the instance table, tensor maps and work lists
    std::vector<char> maps_host(tc_map_bytes());
    std::vector<int> tt(ntc > 0 ? ntc : 1), tf(nf64 > 0 ? nf64 : 1);
    char errbuf[256] = {0};
    for (int k = 0; k < nb; ++k) {
      BatchItem& it = items[k];
      it.st = &states[k];
      char* p = A + inst_off[k];
      if (split) {
        const size_t n2 = (size_t)it.Mp * it.Mp;
        char* maps_dev = p;
        p += al(tc_map_bytes());
        it.X[0] = (float*)p;
        p += al(n2 * 4);
        it.X[1] = (float*)p;
        p += al(n2 * 4);
        it.Sig = (float*)p;
        p += al(n2 * 4);
        it.Xh[0] = p;
        p += al(n2 * 2);
        it.Xl[0] = p;
        p += al(n2 * 2);
        it.Xh[1] = p;
        p += al(n2 * 2);
        it.Xl[1] = p;
        p += al(n2 * 2);
        it.Sh = p;
        p += al(n2 * 2);
        it.Sl = p;
        p += al(n2 * 2);
        if (tc_build_batch_maps(maps_host.data(), it, bf16, errbuf, sizeof errbuf))
          return fail(h, GCP_ERR_CUDA, "gcp_solve_batched: %s", errbuf);
        CK(cudaMemcpy(maps_dev, maps_host.data(), tc_map_bytes(), cudaMemcpyHostToDevice));
        it.maps = maps_dev;
        for (int t = 0; t < it.tc_n; ++t) tt[it.tc_off + t] = k;
      }
      if (!split || mixed) {
        const size_t m2 = (size_t)it.M * it.M;
        for (int i = 0; i < 2; ++i) {
          it.D64[i] = (double*)p;
          p += al(m2 * 8);
        }
        it.S64 = (double*)p;
        p += al(m2 * 8);
        for (int t = 0; t < it.f64_n; ++t) tf[it.f64_off + t] = k;
      }
      if (oz) {
        const size_t n2 = (size_t)it.Mp * it.Mp;
        char* omaps_dev = p;
        p += al(oz_batch_map_bytes());
        for (int sl = 0; sl < kOzSlices; ++sl) {
          it.oz_sl[sl] = p;
          p += al(n2 * 2);
        }
        void** halves[4] = {&it.oz_dh, &it.oz_dl, &it.oz_xh, &it.oz_xl};
        for (int hk = 0; hk < 4; ++hk) {
          *halves[hk] = p;
          p += al(n2 * 2);
        }
        it.oz_rs = (double*)p;
        p += al((size_t)it.Mp * 8);
        it.oz_xs = (double*)p;
        p += al((size_t)it.Mp * 8);
        std::vector<char> om(oz_batch_map_bytes());
        if (oz_build_batch_maps(om.data(), it, errbuf, sizeof errbuf))
          return fail(h, GCP_ERR_CUDA, "gcp_solve_batched: %s", errbuf);
        CK(cudaMemcpy(omaps_dev, om.data(), om.size(), cudaMemcpyHostToDevice));
        it.oz_maps = omaps_dev;
      }
    }
    CK(cudaMemcpy(items_d, items.data(), sizeof(BatchItem) * nb, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(tinst_tc, tt.data(), sizeof(int) * tt.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(tinst_f64, tf.data(), sizeof(int) * tf.size(), cudaMemcpyHostToDevice));
  }

  // Order in which the CTAs take the tensor-core tiles, chosen once per set
  // of instance sizes by timing GEMM1 of the first step (after the guess)
  // with each candidate: (0) the work list's own order, instance after
  // instance; (1) the tiles by estimated cost (tc_tile_cost), largest first,
  // dealt to the CTAs in turn; (2) the same, each round of one tile per CTA
  // dealt in the reverse direction of the one before; (3) instance after
  // instance as in (0), the instances by size, largest first (an instance's
  // tiles stay together, and share their operand panels in L2).  A tile's
  // arithmetic and its partials' place do not depend on the CTA that runs
  // it, so the results are the same under every order.
  const int* order = nullptr;
  if (split && ntc > 0) {
    std::vector<int> tk;
    tk.reserve(nb + 2);
    tk.push_back(h->tune_force);
    tk.push_back(bf16);
    for (int k = 0; k < nb; ++k) tk.push_back(items[k].Mp);
    const bool retune = tk != h->tune_key;
    if (fresh || retune) {
      int dev = 0, nsm = 0;
      CK(cudaGetDevice(&dev));
      CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
      const int G = ntc < nsm ? ntc : nsm;  // CTAs of a launch
      std::vector<int> cost(ntc), lpt(ntc), snake(ntc), bysize;
      bysize.reserve(ntc);
      for (int k = 0; k < nb; ++k)
        for (int t = 0; t < items[k].tc_n; ++t)
          cost[items[k].tc_off + t] = tc_tile_cost(items[k].Mp, t);
      for (int t = 0; t < ntc; ++t) lpt[t] = t;
      std::stable_sort(lpt.begin(), lpt.end(),
                       [&cost](int a, int b) { return cost[a] > cost[b]; });
      for (int t = 0; t < ntc; ++t) {
        const int round = t / G, pos = t % G, r0 = round * G;
        const int width = ntc - r0 < G ? ntc - r0 : G;
        snake[t] = (round & 1) ? lpt[r0 + width - 1 - pos] : lpt[t];
      }
      {
        std::vector<int> inst(nb);
        for (int k = 0; k < nb; ++k) inst[k] = k;
        std::stable_sort(inst.begin(), inst.end(),
                         [&items](int a, int b) { return items[a].Mp > items[b].Mp; });
        for (int k : inst)
          for (int t = 0; t < items[k].tc_n; ++t) bysize.push_back(items[k].tc_off + t);
      }
      const std::vector<int>* cand[4] = {nullptr, &lpt, &snake, &bysize};
      if (retune) {
        int choice = 0;
        double ms[4] = {-1.0, -1.0, -1.0, -1.0};
        if (h->tune_force >= 0) {
          choice = h->tune_force;
        } else if (ntc >= 2 * G) {
          // the first step's state: guess and state set-up as the solve
          // does them (the solve repeats both)
          launch_batch_guess(items_d, nb, maxM, h64, 1, bf16, kSplitScale, gpart, gstride,
                             o.guess, s);
          launch_batch_state_init(items_d, nb, 1, s);
          cudaEvent_t ev[2];
          CK(cudaEventCreate(&ev[0]));
          CK(cudaEventCreate(&ev[1]));
          for (int c = 0; c < 4; ++c) {
            if (c > 0)
              CK(cudaMemcpyAsync(order_d, cand[c]->data(), sizeof(int) * (size_t)ntc,
                                 cudaMemcpyHostToDevice, s));
            const int* oc = c > 0 ? order_d : nullptr;
            bool bad = false;
            for (int rep = 0; rep < 3 && !bad; ++rep) {
              if (rep == 1) CK(cudaEventRecord(ev[0], s));
              bad = tc_launch_batch_gemm(1, items_d, nb, tinst_tc, oc, ntc, part, bf16,
                                         kSplitScale, h->tcs, s) != 0;
            }
            CK(cudaEventRecord(ev[1], s));
            CK(cudaEventSynchronize(ev[1]));
            float t = 0.f;
            if (bad || cudaEventElapsedTime(&t, ev[0], ev[1]) != cudaSuccess) {
              cudaEventDestroy(ev[0]);
              cudaEventDestroy(ev[1]);
              return fail(h, GCP_ERR_CUDA, "batched GEMM1 launch failed (work-order timing)");
            }
            ms[c] = t / 2.0;
            if (ms[c] < ms[choice]) choice = c;
          }
          cudaEventDestroy(ev[0]);
          cudaEventDestroy(ev[1]);
        }
        h->tune_key = tk;
        h->tune_choice = choice;
        for (int c = 0; c < 4; ++c) h->tune_ms[c] = ms[c];
      }
      if (h->tune_choice > 0)
        CK(cudaMemcpyAsync(order_d, cand[h->tune_choice]->data(), sizeof(int) * (size_t)ntc,
                           cudaMemcpyHostToDevice, s));
    }
    if (h->tune_choice > 0) order = order_d;
  }

  Ctl c1{}, c0{};
  c1.stop = c0.stop = o.stop;
  c1.max_iter = c0.max_iter = o.max_iter;
  c1.fixed_iters = c0.fixed_iters = o.fixed_iters;
  c1.tol = c0.tol = o.tol;
  c1.phase = 1;
  c1.final_phase = mixed ? 0 : 1;
  c1.endgame = 1;
  c1.u = kU32;
  c0.phase = 0;
  c0.final_phase = 1;
  c0.endgame = split ? 1 : 0;
  c0.u = kU64;
  c0.mcw_only = oz ? 1 : 0;
  c0.phase_max = mixed ? o.refine_iters : 0;
  // the slice product's dropped digit pairs (the plan of the largest
  // instance, which every instance shares; see oz_weight_cap)
  if (oz && c0.stop == GCP_STOP_IDEMP_FRO) c0.tol -= oz_tail_estimate(maxM, o.tol);
  c1.method = c0.method = o.method;

  auto split_body = [&](cudaGraphConditionalHandle cond, cudaStream_t ss, int use_cond) {
    if (tc_launch_batch_gemm(1, items_d, nb, tinst_tc, order, ntc, part, bf16, kSplitScale,
                             h->tcs, ss))
      return fail(h, GCP_ERR_CUDA, "batched GEMM1 launch failed");
    launch_batch_control(part, items_d, nb, c1, ss);
    if (tc_launch_batch_gemm(2, items_d, nb, tinst_tc, order, ntc, part, bf16, kSplitScale,
                             h->tcs, ss))
      return fail(h, GCP_ERR_CUDA, "batched GEMM2 launch failed");
    launch_batch_any_active(items_d, nb, (unsigned long long)cond, use_cond, active, ss);
    CK(cudaPeekAtLastError());
    return GCP_OK;
  };
  auto f64_body = [&](cudaGraphConditionalHandle cond, cudaStream_t ss, int use_cond) {
    launch_batch_f64_gemm1(items_d, nb, tinst_f64, nf64, part, ss);
    launch_batch_control(part, items_d, nb, c0, ss);
    launch_batch_f64_gemm2(items_d, nb, tinst_f64, nf64, ss);
    launch_batch_any_active(items_d, nb, (unsigned long long)cond, use_cond, active, ss);
    CK(cudaPeekAtLastError());
    return GCP_OK;
  };
  // exact-slice refinement step, as rec_oz_step of a single solve
  auto oz_body = [&](cudaGraphConditionalHandle cond, cudaStream_t ss, int use_cond) {
    launch_batch_oz_slice(items_d, nb, maxM, ss);
    if (launch_batch_oz_gemm(items_d, tinst_tc, ntc, maxM, oz_weight_cap(maxM, o.tol), ss))
      return fail(h, GCP_ERR_CUDA, "batched slice GEMM launch failed");
    launch_batch_oz_finalize(items_d, nb, maxM, part, ss);
    launch_batch_control(part, items_d, nb, c0, ss);
    if (tc_launch_batch_gemm(3, items_d, nb, tinst_tc, order, ntc, part, 0, 1.0f, h->tcs, ss))
      return fail(h, GCP_ERR_CUDA, "batched refinement product launch failed");
    if (c0.stop == GCP_STOP_IDEMP_FRO) {
      // stop test of each new iterate from the split product of K = 3M
      // (as a single solve), instead of a further slice product
      launch_batch_check_halves(items_d, nb, maxM, ss);
      if (tc_launch_batch_gemm(4, items_d, nb, tinst_tc, order, ntc, part, 0, 1.0f, h->tcs, ss))
        return fail(h, GCP_ERR_CUDA, "batched stop-test product launch failed");
      launch_batch_check_control(part, items_d, nb, c0, ss);
    }
    launch_batch_any_active(items_d, nb, (unsigned long long)cond, use_cond, active, ss);
    CK(cudaPeekAtLastError());
    return GCP_OK;
  };
  // one phase: a WHILE node when capturing, else a host loop on the flag
  auto run_phase = [&](auto& body, cudaStream_t ss, bool graph) -> gcp_status {
    if (graph) {
      cudaStreamCaptureStatus cst;
      unsigned long long id = 0;
      cudaGraph_t g = nullptr;
      const cudaGraphNode_t* deps = nullptr;
      const cudaGraphEdgeData* edata = nullptr;
      size_t nd = 0;
      CK(cudaStreamGetCaptureInfo(ss, &cst, &id, &g, &deps, &edata, &nd));
      cudaGraphConditionalHandle cond;
      CK(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
      cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
      p.conditional.handle = cond;
      p.conditional.type = cudaGraphCondTypeWhile;
      p.conditional.size = 1;
      cudaGraphNode_t node;
      CK(cudaGraphAddNode(&node, g, deps, edata, nd, &p));
      cudaGraph_t bodyg = p.conditional.phGraph_out[0];
      CK(cudaStreamUpdateCaptureDependencies(ss, &node, nullptr, 1,
                                             cudaStreamSetCaptureDependencies));
      CK(cudaStreamBeginCaptureToGraph(h->body, bodyg, nullptr, nullptr, 0,
                                       cudaStreamCaptureModeRelaxed));
      gcp_status rr = body(cond, h->body, 1);
      cudaGraph_t outg = nullptr;
      cudaError_t e = cudaStreamEndCapture(h->body, &outg);
      if (rr != GCP_OK) return rr;
      if (e != cudaSuccess) return fail(h, GCP_ERR_CUDA, "body capture: %s", cudaGetErrorString(e));
      return GCP_OK;
    }
    // the control kernel stops every instance by max_iter (fixed_iters)
    // evaluations; the bound here only guards the host loop (64-bit: no
    // overflow for any int option)
    const long long cap = (long long)(o.fixed_iters > 0 ? o.fixed_iters : o.max_iter) + 2;
    for (long long it = 0; it < cap; ++it) {
      gcp_status rr = body(0, ss, 0);
      if (rr != GCP_OK) return rr;
      int hostact = 0;
      CK(cudaMemcpyAsync(&hostact, active, sizeof hostact, cudaMemcpyDeviceToHost, ss));
      CK(cudaStreamSynchronize(ss));
      if (!hostact) break;
    }
    return GCP_OK;
  };
  auto record = [&](cudaStream_t ss, bool graph) -> gcp_status {
    launch_batch_guess(items_d, nb, maxM, h64, split ? 1 : 0, bf16, kSplitScale, gpart, gstride,
                       o.guess, ss);
    launch_batch_state_init(items_d, nb, split ? 1 : 0, ss);
    CK(cudaPeekAtLastError());
    gcp_status rr;
    if (split && (rr = run_phase(split_body, ss, graph)) != GCP_OK) return rr;
    if (mixed) {
      launch_batch_x_to_d64(items_d, nb, maxM, ss);
      launch_batch_phase_begin(items_d, nb, 0, ss);
    }
    if (oz) {
      if ((rr = run_phase(oz_body, ss, graph)) != GCP_OK) return rr;
    } else if ((!split || mixed) && (rr = run_phase(f64_body, ss, graph)) != GCP_OK) {
      return rr;
    }
    launch_batch_copy_out(items_d, nb, maxM, split && !mixed ? 1 : 0, d64, ss);
    launch_batch_energy(items_d, nb, d64, h64, gpart, gstride, ss);
    CK(cudaPeekAtLastError());
    return GCP_OK;
  };
  if (o.use_graph) {
    if (fresh) {
      if (h->bexec) cudaGraphExecDestroy(h->bexec);
      if (h->bgraph) cudaGraphDestroy(h->bgraph);
      h->bexec = nullptr;
      h->bgraph = nullptr;
      h->bkey.clear();
      CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeRelaxed));
      r = record(h->cap, true);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(h->cap, &g);
      if (r != GCP_OK) {
        if (g) cudaGraphDestroy(g);
        return r;
      }
      if (e != cudaSuccess)
        return fail(h, GCP_ERR_CUDA, "batched capture: %s", cudaGetErrorString(e));
      h->bgraph = g;
      CK(cudaGraphInstantiate(&h->bexec, g, 0));
      h->bkey = key;
    }
    CK(cudaGraphLaunch(h->bexec, s));
  } else {
    if ((r = record(s, false)) != GCP_OK) return r;
  }
  std::vector<State> hs(nb);
  CK(cudaMemcpyAsync(hs.data(), states, sizeof(State) * nb, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  gcp_status worst = GCP_OK;
  for (int k = 0; k < nb; ++k) {
    if (hs[k].timeout) return fail(h, GCP_ERR_TIMEOUT, "a device-side wait gave up");
    if (res) {
      fill_result(hs[k], &res[idx[k]]);
      res[idx[k]].energy = hs[k].E;
    }
    if (hs[k].status != GCP_OK && worst == GCP_OK) worst = (gcp_status)hs[k].status;
  }
  if (worst != GCP_OK)
    return fail(h, worst, "gcp_solve_batched: an instance ended with: %s",
                gcp_status_string(worst));
  return GCP_OK;
}

gcp_status gcp_backward(void* hv, const void* H, int M, int N, int ld, int h_dtype,
                        const void* G_D, double g_E, void* dL_dH, const gcp_options* opt) {
  Handle* h = (Handle*)hv;
  if (!h) return GCP_ERR_INVALID_ARG;
  gcp_options o;
  if (opt)
    o = *opt;
  else
    gcp_default_options(&o);
  if (!H || !dL_dH || M <= 0 || N <= 0 || N >= M || ld < M || !valid_dtype(h_dtype) ||
      o.fixed_iters <= 0 || o.ckpt_every < 0 || !(g_E == g_E))
    return fail(h, GCP_ERR_INVALID_ARG,
                "gcp_backward: bad arguments (needs 0 < N < M and opt->fixed_iters > 0)");
  if (o.prec != GCP_FP64 && o.prec != GCP_FP32)
    return fail(h, GCP_ERR_UNSUPPORTED,
                "gcp_backward: the adjoint runs in FP64 or FP32 (prec = GCP_FP64 or GCP_FP32)");
  if (o.guess < GCP_GUESS_CANONICAL || o.guess > GCP_GUESS_HOLE ||
      (o.method != GCP_METHOD_HPCP && o.method != GCP_METHOD_PMCP))
    return fail(h, GCP_ERR_INVALID_ARG, "gcp_backward: bad guess or method");
  if (o.prec == GCP_FP32 && o.method != GCP_METHOD_HPCP)
    return fail(h, GCP_ERR_UNSUPPORTED,
                "gcp_backward: the FP32 adjoint differentiates HPCP steps only");
  cudaStream_t s = (cudaStream_t)o.stream;
  gcp_status r;
  if (o.prec == GCP_FP32) {
    // iterates in the split state, products on the tensor cores
    const int Mp = tc_pad(M);
    size_t nt = tc_num_tiles(Mp);
    if ((size_t)f64_num_tiles(M) > nt) nt = f64_num_tiles(M);
    if ((r = ensure_common(h, nt, M, o.fixed_iters + 2)) != GCP_OK) return r;
    if ((r = ensure_tcs(h)) != GCP_OK) return r;
    char err[256] = {0};
    const int rc = adjoint_backward_tc(&h->adj_tc, H, M, N, ld, h_dtype == GCP_F64, o.guess, G_D,
                                       g_E, dL_dH, o.fixed_iters, o.ckpt_every, h->st, h->part,
                                       h->gpart, h->hist, h->tcs, s, err, sizeof err);
    if (rc != GCP_OK) return fail(h, (gcp_status)rc, "%s", err);
    return GCP_OK;
  }
  if ((r = ensure_common(h, f64_num_tiles(M), M, o.fixed_iters + 2)) != GCP_OK) return r;
  if ((r = ensure_f64(h, M)) != GCP_OK) return r;
  char err[256] = {0};
  const int rc = adjoint_backward(&h->adj, H, M, N, ld, h_dtype == GCP_F64, o.guess, o.method,
                                  G_D, g_E, dL_dH, o.fixed_iters, o.ckpt_every, h->D64[0],
                                  h->D64[1], h->S64, h->part, h->gpart, h->st, h->hist, s, err,
                                  sizeof err);
  if (rc != GCP_OK) return fail(h, (gcp_status)rc, "%s", err);
  return GCP_OK;
}

gcp_status gcp_set_batched_order(void* hv, int order) {
  Handle* h = (Handle*)hv;
  if (!h) return GCP_ERR_INVALID_ARG;
  if (order < -1 || order > 3)
    return fail(h, GCP_ERR_INVALID_ARG, "gcp_set_batched_order: order must be -1, 0, 1, 2 or 3");
  h->tune_force = order;
  return GCP_OK;
}

gcp_status gcp_batched_order(void* hv, int* choice, double* ms) {
  Handle* h = (Handle*)hv;
  if (!h || !choice) return GCP_ERR_INVALID_ARG;
  *choice = h->tune_choice;
  if (ms)
    for (int c = 0; c < 4; ++c) ms[c] = h->tune_ms[c];
  return GCP_OK;
}

// Diagnostic: drive the bounded-wait path of the tensor-core kernel.  One
// split GEMM1 of size M on this handle's workspace (its inputs are whatever
// the buffers hold: only the waits matter), every device-side wait bounded by
// wait_s, and the drain warps first wait on a barrier that no thread arrives
// on.  Every role of the kernel then runs into its bound, records the
// timeout in the state and returns; the kernel frees its TMEM and leaves the
// context usable.
gcp_status gcp_debug_timeout(void* hv, int M, double wait_s, const gcp_options* opt) {
  Handle* h = (Handle*)hv;
  if (!h) return GCP_ERR_INVALID_ARG;
  gcp_options o;
  if (opt)
    o = *opt;
  else
    gcp_default_options(&o);
  if (M <= 0 || !(wait_s > 0.0) || wait_s > 10.0)
    return fail(h, GCP_ERR_INVALID_ARG, "gcp_debug_timeout: bad arguments (0 < wait_s <= 10)");
  cudaStream_t s = (cudaStream_t)o.stream;
  const int Mp = tc_pad(M);
  gcp_status r;
  if ((r = ensure_common(h, tc_num_tiles(Mp), M, 0)) != GCP_OK) return r;
  if ((r = ensure_split(h, Mp, 0)) != GCP_OK) return r;
  State init;
  memset(&init, 0, sizeof init);
  init.theta = 0.25;
  CK(cudaMemcpyAsync(h->st, &init, sizeof init, cudaMemcpyHostToDevice, s));
  const unsigned long long ns = (unsigned long long)(wait_s * 1e9);
  if (tc_launch_gemm1(h->opX[0], h->X[0], h->Sig, h->Sh, h->Sl, M, Mp, nullptr, 1, M, h->part,
                      h->st, 0, kSplitScale, h->tcs, s, ns, 1))
    return fail(h, GCP_ERR_CUDA, "gcp_debug_timeout: launch failed: %s",
                cudaGetErrorString(cudaGetLastError()));
  State hs;
  CK(cudaMemcpyAsync(&hs, h->st, sizeof hs, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  // leave the state as a fresh solve expects it
  memset(&init, 0, sizeof init);
  CK(cudaMemcpyAsync(h->st, &init, sizeof init, cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  if (hs.timeout) return fail(h, GCP_ERR_TIMEOUT, "gcp_debug_timeout: the kernel gave up waiting");
  return GCP_OK;
}

gcp_status gcp_time_kernels(void* hv, int M, int N, int prec, int reps, double* ms,
                            const gcp_options* opt) {
  Handle* h = (Handle*)hv;
  if (!h) return GCP_ERR_INVALID_ARG;
  if (M <= 0 || N <= 0 || N >= M || reps <= 0 || !ms)
    return fail(h, GCP_ERR_INVALID_ARG, "gcp_time_kernels: bad arguments");
  gcp_options o;
  if (opt)
    o = *opt;
  else
    gcp_default_options(&o);
  cudaStream_t s = (cudaStream_t)o.stream;
  const bool split = prec == GCP_FP16X3 || prec == GCP_BF16X3;
  const bool refine = prec == GCP_MIXED_FP16 || prec == GCP_MIXED_BF16;
  if (split) {
    if (h->mp != tc_pad(M) || h->tc_bf16 != (prec == GCP_BF16X3) || !h->opS)
      return fail(h, GCP_ERR_NO_CHECKPOINT, "gcp_time_kernels: no split workspace of this size");
  } else if (refine) {
    if (h->oz_mp != tc_pad(M) || !h->oz_op || h->m64 < M)
      return fail(h, GCP_ERR_NO_CHECKPOINT,
                  "gcp_time_kernels: no slice-refinement workspace of this size");
  } else if (prec == GCP_FP64) {
    if (h->m64 < M) return fail(h, GCP_ERR_NO_CHECKPOINT, "gcp_time_kernels: no FP64 workspace");
  } else {
    return fail(h, GCP_ERR_INVALID_ARG, "gcp_time_kernels: bad prec");
  }
  // a live state: apply = 1 with c = 1/2 (McWeeny coefficients)
  State init;
  memset(&init, 0, sizeof init);
  init.theta = (double)N / (double)M;
  init.apply = 1;
  init.c = 0.5;
  init.a = 0.0;
  init.b = 3.0;
  init.g3 = -2.0;
  init.xshift = 2.0 * init.theta * (1.0 - init.theta) * (init.theta - 0.5);
  CK(cudaMemcpyAsync(h->st, &init, sizeof init, cudaMemcpyHostToDevice, s));
  cudaEvent_t e[4];
  for (int i = 0; i < 4; ++i) CK(cudaEventCreate(&e[i]));
  const int Mp = h->mp, bf = h->tc_bf16;
  CK(cudaEventRecord(e[0], s));
  for (int r = 0; r < reps; ++r) {
    if (refine) {
      if (launch_oz_gemm(h->oz_op, h->oz_rscale, h->S64, M, h->oz_mp, oz_weight_cap(M, o.tol),
                         h->st, s))
        return fail(h, GCP_ERR_CUDA, "slice GEMM launch failed");
    } else if (split) {
      if (tc_launch_gemm1(h->opX[0], h->X[0], h->Sig, h->Sh, h->Sl, M, Mp, nullptr, 1, M, h->part,
                          h->st, bf, kSplitScale, h->tcs, s))
        return fail(h, GCP_ERR_CUDA, "GEMM1 launch failed");
    } else {
      launch_f64_gemm1(h->D64[0], h->S64, M, M, nullptr, 1, M, h->part, h->st, s);
    }
  }
  CK(cudaEventRecord(e[1], s));
  CK(cudaEventRecord(e[2], s));
  for (int r = 0; r < reps; ++r) {
    if (refine) {
      if (tc_launch_mcweeny64(h->oz_opX, h->oz_opD, h->S64, h->D64[0], h->D64[1], h->oz_xscale,
                              h->oz_rscale, M, h->oz_mp, h->st, h->tcs, s))
        return fail(h, GCP_ERR_CUDA, "refinement product launch failed");
    } else if (split) {
      if (tc_launch_gemm2(h->opS, h->opX[0], h->X[0], h->Sig, h->X[1], h->Xh[1], h->Xl[1], M, Mp,
                          h->st, bf, kSplitScale, h->tcs, s))
        return fail(h, GCP_ERR_CUDA, "GEMM2 launch failed");
    } else {
      launch_f64_gemm2(h->S64, h->D64[0], h->D64[1], M, M, h->st, s);
    }
  }
  CK(cudaEventRecord(e[3], s));
  CK(cudaEventSynchronize(e[3]));
  float t1 = 0.f, t2 = 0.f, t3 = 0.f;
  CK(cudaEventElapsedTime(&t1, e[0], e[1]));
  CK(cudaEventElapsedTime(&t2, e[2], e[3]));
  if (refine) {
    // the stop-test product of the step (reuses the first two events)
    CK(cudaEventRecord(e[0], s));
    for (int r = 0; r < reps; ++r)
      if (tc_launch_check(h->oz_opD, h->oz_opX, h->oz_emaps, h->S64, h->D64[1], h->part, M,
                          h->oz_mp, h->st, h->tcs, s))
        return fail(h, GCP_ERR_CUDA, "stop-test product launch failed");
    CK(cudaEventRecord(e[1], s));
    CK(cudaEventSynchronize(e[1]));
    CK(cudaEventElapsedTime(&t3, e[0], e[1]));
  }
  for (int i = 0; i < 4; ++i) cudaEventDestroy(e[i]);
  ms[0] = t1 / reps;
  ms[1] = t2 / reps;
  if (refine) {
    ms[2] = t3 / reps;
    ms[3] = (double)oz_num_products(M, oz_weight_cap(M, o.tol));
  }
  State hs;
  CK(cudaMemcpy(&hs, h->st, sizeof hs, cudaMemcpyDeviceToHost));
  if (hs.timeout) return fail(h, GCP_ERR_TIMEOUT, "a device-side wait gave up");
  return GCP_OK;
}

}  // extern "C"
