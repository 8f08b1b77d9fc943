// Device-side control of the recursion: one single-block kernel per step
// reduces the GEMM1 partials (in tile order, so the sums are deterministic),
// applies the stop tests, computes c_n (Eq. mcwgamb) and the coefficients of
// the cubic update (Eq. hpcp3), and sets the CUDA-graph WHILE condition, so
// a whole solve runs without a host round trip.  Plus the small conversion
// kernels around the loop.
//
// Stop rules (readings where the paper is silent, shared with the oracle):
//   * ||D^2 - D||_F <= tol or Tr(D - D^2) <= tol (the paper's test);
//   * 0/0 guard: when |Tr(D - D^2)| <= 16 M u max(1, Tr D) and the stop
//     test still fails, the FP64 step is a McWeeny step (c = 1/2, the limit
//     of the recursion as gamma -> 0, Eq. mcweeny3) and the split phase
//     ends; in fixed-iteration mode the step becomes an identity step;
//   * c_0 outside [0,1] reports GCP_ERR_ILL_CONDITIONED (Eqs. pmcpcons2-3);
//   * FP64 stagnation: once R < 1e-8, two consecutive non-decreasing R;
//   * split-precision floor: once R < 1e-2, a step that fails to reduce R
//     by 4x ends the split phase (the products can go no further);
//   * mixed modes with the ||D^2 - D||_F test: the split phase also ends
//     once R <= sqrt(tol/3)/2, from where one refinement step suffices.
#include "gcp_device.cuh"
#include "gcp_internal.cuh"

namespace gcp {

namespace {
constexpr int kCtlThreads = 256;

// One control decision from the summed partials v of the iterate's GEMM1.
// Returns 1 when the phase stops for this state (already stopped included).
// Coefficients of D+ = a D + b S + g3 S D for c and the method, and the J
// coefficient of the shifted update X+ = D+ - theta J (split phase):
//   HPCP (Eq. hpcp3): a = 1 - 2c, b = 2 + 2c, g3 = -2,
//     xshift = 2 theta (1 - theta)(theta - c);
//   PMCP (Eq. pm1): c <= 1/2: a = (1-2c)/(1-c), b = (1+c)/(1-c), g3 = -1/(1-c);
//     c > 1/2: a = 0, b = (1+c)/c, g3 = -1/c;
//     xshift = a theta + b theta^2 + g3 theta^3 - theta.
// Both give the McWeeny step (Eq. mcweeny3) at c = 1/2.
__device__ void set_coeffs(State* st, double c, int method) {
  const double th = st->theta;
  st->c = c;
  if (method == GCP_METHOD_PMCP) {
    double a, b, g3;
    if (c <= 0.5) {
      a = (1.0 - 2.0 * c) / (1.0 - c);
      b = (1.0 + c) / (1.0 - c);
      g3 = -1.0 / (1.0 - c);
    } else {
      a = 0.0;
      b = (1.0 + c) / c;
      g3 = -1.0 / c;
    }
    st->a = a;
    st->b = b;
    st->g3 = g3;
    st->xshift = a * th + b * th * th + g3 * th * th * th - th;
  } else {
    st->a = 1.0 - 2.0 * c;
    st->b = 2.0 + 2.0 * c;
    st->g3 = -2.0;
    st->xshift = 2.0 * th * (1.0 - th) * (th - c);
  }
}

__device__ int control_decide(const double (&v)[5], State* st, double* hist, const Ctl& ctl) {
  if (st->stopped) return 1;
  // FP64 phase: v = (Tr D, Tr S, sum S o D, R^2, E).
  // Split phase, on D = theta J + X and S = theta^2 J + Sigma (J the identity
  // on the unpadded block): v = (Tr X, Tr Sigma, sum Sigma o X, R^2, E) and
  //   Tr D = theta M + Tr X,  Tr S = theta^2 M + Tr Sigma,
  //   sum S o D = theta^3 M + theta^2 Tr X + theta Tr Sigma + sum Sigma o X;
  // den and num are formed from these parts directly, which keeps the O(M)
  // constant terms out of the cancellation near convergence.
  double T1, T2, T3, den, num;
  if (ctl.phase == 1) {
    const double th = st->theta, thb = 1.0 - th, Md = (double)ctl.M;
    T1 = th * Md + v[0];
    T2 = th * th * Md + v[1];
    T3 = th * th * th * Md + th * th * v[0] + th * v[1] + v[2];
    den = th * thb * Md + v[0] - v[1];
    num = th * th * thb * Md + thb * v[1] - th * th * v[0] - v[2];
  } else {
    T1 = v[0];
    T2 = v[1];
    T3 = v[2];
    den = T1 - T2;
    num = T2 - T3;
  }
  const double R = sqrt(fmax(v[3], 0.0)), E = v[4];
  st->T1 = T1;
  st->T2 = T2;
  st->T3 = T3;
  st->R = R;
  st->E = E;
  const int n = st->n;
  double* rec = nullptr;
  if (hist && st->hist_n < ctl.hist_cap) {
    rec = hist + (size_t)st->hist_n * GCP_HISTORY_FIELDS;
    rec[0] = n;
    rec[1] = T1;
    rec[2] = T2;
    rec[3] = T3;
    rec[4] = R;
    rec[5] = __longlong_as_double(0x7ff8000000000000ll);
    rec[6] = E;
    rec[7] = ctl.phase;
    st->hist_n += 1;
  }
  // kind: 1 converged, 2 split-precision floor, 3 terminal
  int stop = 0, status = GCP_OK, kind = 0;
  if (st->timeout) {
    stop = 1;
    kind = 3;
    status = GCP_ERR_TIMEOUT;
  } else if (!isfinite(T1) || !isfinite(T2) || !isfinite(T3) || !isfinite(R)) {
    stop = 1;
    kind = 3;
    status = GCP_ERR_NONFINITE;
  } else if (ctl.fixed_iters > 0) {
    if (n >= ctl.fixed_iters) {
      stop = 1;
      kind = 1;
    }
  } else {
    const double crit = (ctl.stop == GCP_STOP_IDEMP_FRO) ? R : fabs(den);
    if (crit <= ctl.tol) {
      stop = 1;
      kind = 1;
    } else if (ctl.phase == 0 && ((R < 1e-8 && R >= st->Rp0 && st->Rp0 >= st->Rp1) ||
                                  (ctl.mcw_only && R > 0.5 * st->Rp0))) {
      // stagnation (the slice refinement: a step that does not halve R has
      // reached the accuracy of its products)
      stop = 1;
      kind = 3;
      status = (R <= ctl.tol) ? GCP_OK : GCP_ERR_NOT_CONVERGED;
    } else if (ctl.phase == 1 && R < 1e-2 && R > 0.25 * st->Rp0) {
      // the split products can go no further: the residual stalls
      stop = 1;
      kind = 2;
    } else if (ctl.phase == 1 && !ctl.final_phase && ctl.stop == GCP_STOP_IDEMP_FRO &&
               R <= 0.5 * sqrt(ctl.tol / 3.0)) {
      // mixed modes: one McWeeny step of the refinement takes R to ~3 R^2,
      // below tol/12 from here, so the split phase hands over now instead of
      // running on to its floor
      stop = 1;
      kind = 2;
    } else if (n >= ctl.max_iter || (ctl.phase_max > 0 && n - st->n_phase0 >= ctl.phase_max)) {
      // max_iter, or the step cap of this phase (refine_iters)
      stop = 1;
      kind = 3;
      status = GCP_ERR_NOT_CONVERGED;
    }
  }
  // Endgame of the split and refinement phases (ctl.endgame): once
  // R < 0.05 every eigenvalue of D lies within ~R of 0 or 1, and c is set
  // to 1/2, the McWeeny step (Eq. mcweeny3) that HPCP itself reaches as
  // gamma -> 0.  The quotient of Eq. mcwgamb would be a ratio of two
  // vanishing traces polluted by the rounding of the tensor-core products;
  // the McWeeny step needs neither, and because it does not conserve the
  // trace it also removes the rounding drift of Tr D (the eigenvalues go to
  // exactly 0 or 1).  The same switch applies while that drift is not small
  // against Tr(D - D^2).  The plain FP64 path keeps the oracle's rule.
  //
  // Fixed-iteration split phase (the recursion gcp_backward differentiates
  // in FP32): the same c_n rules, and where a free-running solve would stop
  // at the floor of its products (the stall rule above), every remaining
  // step is an identity step.  Without the trace-restoring c and the
  // endgame, the truncating FP32 accumulation of the tensor cores lets
  // Tr D drift by ~M 1e-7 per step, c_n leaves [0, 1] once Tr(D - D^2) is
  // of that size, and the iterate stalls far above the floor.
  const bool fixed_split = ctl.phase == 1 && ctl.fixed_iters > 0;
  const bool mcw = ctl.mcw_only || ctl.endgame && (ctl.fixed_iters == 0 || fixed_split) &&
                   (R < 0.05 || fabs(T1 - (double)ctl.N) > 0.05 * fabs(den));
  int* kind_out = (ctl.step_kind && fixed_split && n < ctl.fixed_iters) ? ctl.step_kind + n
                                                                         : nullptr;
  if (kind_out) *kind_out = kStepIdentity;
  if (!stop && fixed_split &&
      (st->split_floor || (ctl.endgame && R < 1e-2 && R > 0.25 * st->Rp0))) {
    st->split_floor = 1;
    st->apply = 0;  // identity step
    st->n = n + 1;
    st->parity ^= 1;
  } else if (!stop) {
    // 0/0 guard.  FP64: 16 M u max(1, Tr D) (as in the oracle).  Split phase:
    // the noise of den is set by the FP32 rounding of the O(1) diagonal,
    // 16 sqrt(M) u_32.
    const double den_min = ctl.phase == 1 ? 16.0 * sqrt((double)ctl.M) * ctl.u
                                          : 16.0 * (double)ctl.M * ctl.u * fmax(1.0, T1);
    // Refinement endgame: the McWeeny step leaves Tr D+ = 3 T2 - 2 T3, off N
    // by the second-order imbalance of the eigenvalue errors (up to ~3 R^2).
    // The step of Eq. hpcp3 with 1 - 2c = (N - 3 T2 + 2 T3) / (T1 - T2) has
    // Tr D+ = N exactly; it is taken when that c lies within 1/2 +- 0.05,
    // where it converges like the McWeeny step.  Near idempotency the
    // eigenvalues sit on both sides of 0 and 1, so T1 - T2 may be negative.
    double c_mcw = 0.5;
    if (mcw && ctl.phase == 0 && ctl.endgame && fabs(den) > den_min) {
      const double g = ((double)ctl.N - (3.0 * T2 - 2.0 * T3)) / den;
      if (fabs(g) <= 0.1) c_mcw = 0.5 * (1.0 - g);
    }
    if (fabs(den) <= den_min && !mcw) {
      if (ctl.fixed_iters > 0) {
        st->apply = 0;  // identity step (kind_out already says so)
        st->n = n + 1;
        st->parity ^= 1;
      } else if (R <= ctl.tol) {
        stop = 1;
        kind = 1;
      } else if (ctl.phase == 1) {
        stop = 1;
        kind = 2;
      } else {
        // FP64, Tr(D - D^2) at rounding level but R > tol: McWeeny step
        // (c = 1/2), as in the oracle; the stagnation rule ends a loop that
        // can go no further
        set_coeffs(st, 0.5, GCP_METHOD_HPCP);
        st->apply = 1;
        st->Rp1 = st->Rp0;
        st->Rp0 = R;
        st->n = n + 1;
        st->parity ^= 1;
        if (rec) rec[5] = 0.5;
      }
    } else {
      // Split phase (before the endgame): c also absorbs the FP32 rounding
      // drift of the trace, so that Tr D_{n+1} = N for the traces as
      // computed (exact arithmetic gives Tr D_n = N and the plain
      // Eq. mcwgamb): with delta = Tr D - N, HPCP takes
      // c = (num + delta/2) / den; PMCP (Eq. pm1) c = (num + delta)/(den +
      // delta) on its c <= 1/2 branch and num / (den - delta) on the other.
      // FP64: Eq. mcwgamb.
      double c;
      if (mcw) {
        c = c_mcw;
      } else if (ctl.phase == 1) {
        const double dl = T1 - (double)ctl.N;
        if (ctl.method == GCP_METHOD_PMCP)
          c = (num / den <= 0.5) ? (num + dl) / (den + dl) : num / (den - dl);
        else
          c = (num + 0.5 * dl) / den;
      } else {
        c = num / den;
      }
      const int method = mcw ? (int)GCP_METHOD_HPCP : ctl.method;
      if (n == 0 && !(c >= 0.0 && c <= 1.0) && ctl.fixed_iters == 0) {
        stop = 1;
        kind = 3;
        status = GCP_ERR_ILL_CONDITIONED;
      } else if (ctl.endgame && n > 0 && !(c >= -0.05 && c <= 1.05) &&
                 (ctl.fixed_iters == 0 || fixed_split)) {
        // c left the stable domain (rounding noise): McWeeny step instead
        set_coeffs(st, 0.5, GCP_METHOD_HPCP);
        st->apply = 1;
        st->Rp1 = st->Rp0;
        st->Rp0 = R;
        st->n = n + 1;
        if (ctl.phase == 1) st->n_lowp += 1;
        st->parity ^= 1;
        if (rec) rec[5] = 0.5;
        if (kind_out) *kind_out = kStepMcWeeny;
      } else {
        set_coeffs(st, c, method);
        st->apply = 1;
        st->Rp1 = st->Rp0;
        st->Rp0 = R;
        st->n = n + 1;
        if (ctl.phase == 1) st->n_lowp += 1;
        st->parity ^= 1;
        if (rec) rec[5] = c;
        if (kind_out) *kind_out = mcw ? kStepMcWeeny : kStepRestoring;
      }
    }
  }
  if (stop) {
    st->stopped = 1;
    st->apply = 0;
    if (kind == 1) {
      st->converged = 1;
      st->status = GCP_OK;
    } else if (kind == 3) {
      st->terminal = 1;
      st->status = status;
    } else {
      st->lowp_done = 1;
      if (ctl.final_phase) {
        st->terminal = 1;
        st->status = GCP_ERR_NOT_CONVERGED;
      }
    }
  }
  return stop;
}

__global__ void __launch_bounds__(kCtlThreads) control_kernel(const double* __restrict__ part,
                                                              int ntiles, State* st, double* hist,
                                                              Ctl ctl,
                                                              cudaGraphConditionalHandle cond,
                                                              int use_cond) {
  __shared__ double red[32 * 5];
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
    const double* p = part + (size_t)t * kPartFields;
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] += p[k];
  }
  block_sum<5>(v, red);
  if (threadIdx.x != 0) return;
  const int stop = control_decide(v, st, hist, ctl);
  if (use_cond) cudaGraphSetConditional(cond, stop ? 0u : 1u);
}

// Stop test after a refinement step D -> D1, from the check product's
// per-tile partials (Tr D1, Tr D1^2, -, R1^2): the iterate the next step
// would evaluate exactly is accepted now when R1 = ||D1^2 - D1||_F <= tol.
// Otherwise nothing changes and the next step evaluates D1 with the exact
// product (and stops there if the two disagree about tol).  The WHILE
// condition is set after this kernel as after the step's control kernel.
__device__ void check_decide(const double (&v)[5], State* st, double* hist, const Ctl& ctl) {
  if (!st->stopped && !st->timeout) {
    const double T1 = v[0], T2 = v[1], R = sqrt(fmax(v[3], 0.0));
    if (isfinite(T1) && isfinite(T2) && isfinite(R) && R <= ctl.tol) {
      st->T1 = T1;
      st->T2 = T2;
      st->T3 = __longlong_as_double(0x7ff8000000000000ll);  // not evaluated
      st->R = R;
      st->stopped = 1;
      st->apply = 0;
      st->converged = 1;
      st->status = GCP_OK;
      if (hist && st->hist_n < ctl.hist_cap) {
        double* rec = hist + (size_t)st->hist_n * GCP_HISTORY_FIELDS;
        rec[0] = st->n;
        rec[1] = T1;
        rec[2] = T2;
        rec[3] = st->T3;
        rec[4] = R;
        rec[5] = st->T3;
        rec[6] = st->E;
        rec[7] = ctl.phase;
        st->hist_n += 1;
      }
    }
  }
}

__global__ void __launch_bounds__(kCtlThreads) check_control_kernel(
    const double* __restrict__ part, int ntiles, State* st, double* hist, Ctl ctl,
    cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ double red[32 * 5];
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (!st->stopped)
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
      const double* p = part + (size_t)t * kPartFields;
#pragma unroll
      for (int k = 0; k < 5; ++k) v[k] += p[k];
    }
  block_sum<5>(v, red);
  if (threadIdx.x != 0) return;
  check_decide(v, st, hist, ctl);
  if (use_cond) cudaGraphSetConditional(cond, st->stopped ? 0u : 1u);
}

// Batched stop test after a refinement step: block b sums instance b's
// tensor-core tile partials in the order of a single solve's
// check_control_kernel and takes the same decision.
__global__ void __launch_bounds__(kCtlThreads) batch_check_control_kernel(
    const double* __restrict__ part, const BatchItem* items, Ctl ctl) {
  __shared__ double red[32 * 5];
  const BatchItem& it = items[blockIdx.x];
  State* st = it.st;
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (!st->stopped)
    for (int t = threadIdx.x; t < it.tc_n; t += blockDim.x) {
      const double* p = part + (size_t)(it.tc_off + t) * kPartFields;
#pragma unroll
      for (int k = 0; k < 5; ++k) v[k] += p[k];
    }
  block_sum<5>(v, red);
  if (threadIdx.x != 0) return;
  Ctl c = ctl;
  c.M = it.M;
  c.N = it.N;
  check_decide(v, st, nullptr, c);
}

// Batched control: block b decides for instance b from its own tiles'
// partial sums (per-instance c_n and stop mask).
__global__ void __launch_bounds__(kCtlThreads) batch_control_kernel(const double* __restrict__ part,
                                                                    const BatchItem* items,
                                                                    Ctl ctl) {
  __shared__ double red[32 * 5];
  const BatchItem& it = items[blockIdx.x];
  // partial-sum slots: the tensor-core tiles (split phase), the FP64 tiles,
  // or the exact-slice finalize blocks (refinement with mcw_only)
  const int off = ctl.phase == 1 ? it.tc_off : (ctl.mcw_only ? it.oz_off : it.f64_off);
  const int n = ctl.phase == 1 ? it.tc_n : (ctl.mcw_only ? oz_finalize_blocks(it.M) : it.f64_n);
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const double* p = part + (size_t)(off + t) * kPartFields;
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] += p[k];
  }
  block_sum<5>(v, red);
  if (threadIdx.x != 0) return;
  Ctl c = ctl;
  c.M = it.M;
  c.N = it.N;
  control_decide(v, it.st, nullptr, c);
}

// WHILE condition of a batched phase: continue while any instance runs.
__global__ void batch_any_active_kernel(const BatchItem* items, int batch,
                                        cudaGraphConditionalHandle cond, int use_cond,
                                        int* active_out) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < batch; b += blockDim.x)
    if (!items[b].st->stopped) atomicOr(&any, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (active_out) *active_out = any;
    if (use_cond) cudaGraphSetConditional(cond, any ? 1u : 0u);
  }
}

__device__ void state_init_dev(State* st, int phase);
__device__ void phase_begin_dev(State* st, int phase);

__global__ void state_init_kernel(State* st, int phase) { state_init_dev(st, phase); }
__global__ void phase_begin_kernel(State* st, int phase) { phase_begin_dev(st, phase); }
__global__ void batch_state_init_kernel(const BatchItem* items, int batch, int phase) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < batch) state_init_dev(items[b].st, phase);
}
__global__ void batch_phase_begin_kernel(const BatchItem* items, int batch, int phase) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < batch) phase_begin_dev(items[b].st, phase);
}

__device__ void state_init_dev(State* st, int phase) {
  // zero everything except the guess parameters written just before
  st->n = 0;
  st->n_lowp = 0;
  st->stopped = 0;
  st->status = GCP_OK;
  st->apply = 0;
  st->parity = 0;
  st->phase = phase;
  st->lowp_done = 0;
  st->timeout = 0;
  st->hist_n = 0;
  st->converged = 0;
  st->terminal = 0;
  st->n_phase0 = 0;
  st->split_floor = 0;
  if (st->no_gap) {  // D = theta I, nothing to iterate
    st->stopped = 1;
    st->terminal = 1;
    st->status = GCP_ERR_NO_GAP;
  }
  st->c = __longlong_as_double(0x7ff8000000000000ll);
  st->a = st->b = 0.0;
  st->g3 = -2.0;
  st->T1 = st->T2 = st->T3 = st->R = st->E = 0.0;
  st->Rp0 = st->Rp1 = INFINITY;
  st->xshift = 0.0;
}

__device__ void phase_begin_dev(State* st, int phase) {
  // the FP64 refinement runs only after a split phase that reached its floor
  const int go = st->lowp_done && !st->converged && !st->terminal && !st->no_gap;
  st->stopped = go ? 0 : 1;
  st->phase = phase;
  st->parity = 0;
  st->n_phase0 = st->n;
  st->Rp0 = st->Rp1 = INFINITY;
}

template <typename O>
__global__ void copy_out_f64_kernel(const double* __restrict__ b0, const double* __restrict__ b1,
                                    const State* __restrict__ st, int M, int ld,
                                    O* __restrict__ out, int ldo) {
  const double* src = st->parity ? b1 : b0;
  const int i = blockIdx.y;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x)
    out[(size_t)i * ldo + j] = (O)src[(size_t)i * ld + j];
}

template <typename O>
__global__ void copy_out_x_kernel(const float* __restrict__ X0, const float* __restrict__ X1,
                                  const State* __restrict__ st, int M, int ldx, O* __restrict__ out,
                                  int ldo) {
  const float* src = st->parity ? X1 : X0;
  const double th = st->theta;
  const int i = blockIdx.y;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
    double v = (double)src[(size_t)i * ldx + j];
    if (i == j) v += th;
    out[(size_t)i * ldo + j] = (O)v;
  }
}

__global__ void x_to_d64_kernel(const float* __restrict__ X0, const float* __restrict__ X1,
                                const State* __restrict__ st, int M, int ldx, double* __restrict__ D,
                                int ldd) {
  const float* src = st->parity ? X1 : X0;
  const double th = st->theta;
  const int i = blockIdx.y;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
    // upper-triangle value for both (i, j) and (j, i): exactly symmetric
    double v = (double)src[(size_t)(i < j ? i : j) * ldx + (i < j ? j : i)];
    if (i == j) v += th;
    D[(size_t)i * ldd + j] = v;
  }
}

template <typename I, typename O>
__global__ void convert_kernel(const I* __restrict__ in, int ldi, O* __restrict__ out, int ldo,
                               int M) {
  const int i = blockIdx.y;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x)
    out[(size_t)i * ldo + j] = (O)in[(size_t)i * ldi + j];
}

template <typename O>
__global__ void fill_kernel(O* __restrict__ out, int M, int ldo, double diag) {
  const int i = blockIdx.y;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x)
    out[(size_t)i * ldo + j] = (O)(i == j ? diag : 0.0);
}

template <typename I, bool BF16>
__global__ void d_to_x_kernel(const I* __restrict__ D, int M, int ld, float* __restrict__ X,
                              typename Split<BF16>::T* __restrict__ Xh,
                              typename Split<BF16>::T* __restrict__ Xl, int Mp, float scale,
                              double theta) {
  const int i = blockIdx.y;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < Mp; j += gridDim.x * blockDim.x) {
    double v = 0.0;
    if (i < M && j < M) {
      // the upper triangle of D only (exactly symmetric split state)
      v = (double)(i <= j ? D[(size_t)i * ld + j] : D[(size_t)j * ld + i]);
      if (i == j) v -= theta;
    }
    const float x = (float)v;
    const size_t o = (size_t)i * Mp + j;
    X[o] = x;
    typename Split<BF16>::T h, l;
    Split<BF16>::split(x * scale, h, l);
    Xh[o] = h;
    Xl[o] = l;
  }
}

inline dim3 row_grid(int cols, int rows) {
  int gx = (cols + 255) / 256;
  if (gx > 8) gx = 8;
  return dim3(gx, rows);
}
}  // namespace

void launch_control(const double* part, int ntiles, State* st, double* hist, Ctl ctl,
                    unsigned long long cond_handle, int use_cond, cudaStream_t s) {
  control_kernel<<<1, kCtlThreads, 0, s>>>(part, ntiles, st, hist, ctl,
                                           (cudaGraphConditionalHandle)cond_handle, use_cond);
}

void launch_check_control(const double* part, int ntiles, State* st, double* hist, Ctl ctl,
                          unsigned long long cond_handle, int use_cond, cudaStream_t s) {
  check_control_kernel<<<1, kCtlThreads, 0, s>>>(part, ntiles, st, hist, ctl,
                                                 (cudaGraphConditionalHandle)cond_handle,
                                                 use_cond);
}

void launch_state_init(State* st, int phase, cudaStream_t s) {
  state_init_kernel<<<1, 1, 0, s>>>(st, phase);
}

void launch_phase_begin(State* st, int phase, cudaStream_t s) {
  phase_begin_kernel<<<1, 1, 0, s>>>(st, phase);
}

void launch_copy_out_f64(const double* b0, const double* b1, const State* st, int M, int ld,
                         void* out, int out_f64, int ldo, cudaStream_t s) {
  if (out_f64)
    copy_out_f64_kernel<double><<<row_grid(M, M), 256, 0, s>>>(b0, b1, st, M, ld, (double*)out, ldo);
  else
    copy_out_f64_kernel<float><<<row_grid(M, M), 256, 0, s>>>(b0, b1, st, M, ld, (float*)out, ldo);
}

void launch_copy_out_x(const float* X0, const float* X1, const State* st, int M, int ldx,
                       void* out, int out_f64, int ldo, cudaStream_t s) {
  if (out_f64)
    copy_out_x_kernel<double><<<row_grid(M, M), 256, 0, s>>>(X0, X1, st, M, ldx, (double*)out, ldo);
  else
    copy_out_x_kernel<float><<<row_grid(M, M), 256, 0, s>>>(X0, X1, st, M, ldx, (float*)out, ldo);
}

void launch_x_to_d64(const float* X0, const float* X1, State* st, int M, int ldx, double* D,
                     int ldd, cudaStream_t s) {
  x_to_d64_kernel<<<row_grid(M, M), 256, 0, s>>>(X0, X1, st, M, ldx, D, ldd);
}

void launch_d_to_x(const void* D, int d_f64, int M, int ld, float* X, void* Xh, void* Xl, int Mp,
                   int bf16, float split_scale, double theta, cudaStream_t s) {
  const dim3 g = row_grid(Mp, Mp);
  if (bf16) {
    using T = Split<true>::T;
    if (d_f64)
      d_to_x_kernel<double, true><<<g, 256, 0, s>>>((const double*)D, M, ld, X, (T*)Xh, (T*)Xl, Mp,
                                                   split_scale, theta);
    else
      d_to_x_kernel<float, true><<<g, 256, 0, s>>>((const float*)D, M, ld, X, (T*)Xh, (T*)Xl, Mp,
                                                  split_scale, theta);
  } else {
    using T = Split<false>::T;
    if (d_f64)
      d_to_x_kernel<double, false><<<g, 256, 0, s>>>((const double*)D, M, ld, X, (T*)Xh, (T*)Xl,
                                                    Mp, split_scale, theta);
    else
      d_to_x_kernel<float, false><<<g, 256, 0, s>>>((const float*)D, M, ld, X, (T*)Xh, (T*)Xl, Mp,
                                                   split_scale, theta);
  }
}

void launch_fill(const void*, void* out, int out_f64, int M, int ldo, double diag, cudaStream_t s) {
  if (out_f64)
    fill_kernel<double><<<row_grid(M, M), 256, 0, s>>>((double*)out, M, ldo, diag);
  else
    fill_kernel<float><<<row_grid(M, M), 256, 0, s>>>((float*)out, M, ldo, diag);
}

void launch_convert(const void* in, int in_f64, int ldi, void* out, int out_f64, int ldo, int M,
                    cudaStream_t s) {
  const dim3 g = row_grid(M, M);
  if (in_f64 && out_f64)
    convert_kernel<double, double><<<g, 256, 0, s>>>((const double*)in, ldi, (double*)out, ldo, M);
  else if (in_f64)
    convert_kernel<double, float><<<g, 256, 0, s>>>((const double*)in, ldi, (float*)out, ldo, M);
  else if (out_f64)
    convert_kernel<float, double><<<g, 256, 0, s>>>((const float*)in, ldi, (double*)out, ldo, M);
  else
    convert_kernel<float, float><<<g, 256, 0, s>>>((const float*)in, ldi, (float*)out, ldo, M);
}

}  // namespace gcp

// ---- energy E = Tr(H D) = sum_ij D_ij H_ij of the returned D -------------
namespace gcp {
namespace {
template <typename DT, typename HT>
__global__ void __launch_bounds__(256) energy_kernel(const DT* __restrict__ D, int ldd,
                                                     const HT* __restrict__ H, int ldh, int M,
                                                     double* __restrict__ part) {
  __shared__ double red[32];
  double v[1] = {0.0};
  const int warps = blockDim.x / 32;
  const int gw = blockIdx.x * warps + (threadIdx.x >> 5), nw = gridDim.x * warps;
  const int lane = threadIdx.x & 31;
  for (int i = gw; i < M; i += nw) {
    const DT* d = D + (size_t)i * ldd;
    const HT* hr = H + (size_t)i * ldh;
    for (int j = lane; j < M; j += 32) v[0] += (double)d[j] * (double)hr[j];
  }
  block_sum<1>(v, red);
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
}

__global__ void energy_finalize_kernel(const double* __restrict__ part, int nb, State* st) {
  if (threadIdx.x != 0) return;
  double e = 0.0;
  for (int b = 0; b < nb; ++b) e += part[b];
  st->E = e;
}
}  // namespace

void launch_energy(const void* D, int d_f64, int ldd, const void* H, int h_f64, int ldh, int M,
                   double* part, State* st, cudaStream_t s) {
  const int nb = guess_partial_blocks(M);
  if (d_f64 && h_f64)
    energy_kernel<double, double><<<nb, 256, 0, s>>>((const double*)D, ldd, (const double*)H, ldh,
                                                    M, part);
  else if (d_f64)
    energy_kernel<double, float><<<nb, 256, 0, s>>>((const double*)D, ldd, (const float*)H, ldh, M,
                                                   part);
  else if (h_f64)
    energy_kernel<float, double><<<nb, 256, 0, s>>>((const float*)D, ldd, (const double*)H, ldh, M,
                                                   part);
  else
    energy_kernel<float, float><<<nb, 256, 0, s>>>((const float*)D, ldd, (const float*)H, ldh, M,
                                                  part);
  energy_finalize_kernel<<<1, 32, 0, s>>>(part, nb, st);
}

// ---- batched elementwise kernels (grid.y = instance) ---------------------
// Each block (x, instance) strides over the instance's M x M elements, so
// that a small instance costs a few blocks instead of one per row of the
// largest.
namespace {
__global__ void batch_x_to_d64_kernel(const BatchItem* items) {
  const BatchItem& it = items[blockIdx.y];
  const float* src = it.st->parity ? it.X[1] : it.X[0];
  const double th = it.st->theta;
  const size_t n = (size_t)it.M * it.M;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / it.M), j = (int)(e % it.M);
    double v = (double)src[(size_t)(i < j ? i : j) * it.Mp + (i < j ? j : i)];
    if (i == j) v += th;
    it.D64[0][e] = v;
  }
}

template <typename O>
__global__ void batch_copy_out_kernel(const BatchItem* items, int from_x) {
  const BatchItem& it = items[blockIdx.y];
  O* out = (O*)it.D_out;
  const int p = it.st->parity;
  const size_t n = (size_t)it.M * it.M;
  const float* srcx = it.X[p];
  const double* srcd = it.D64[p];
  const double th = it.st->theta;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / it.M), j = (int)(e % it.M);
    double v;
    if (from_x) {
      v = (double)srcx[(size_t)i * it.Mp + j];
      if (i == j) v += th;
    } else {
      v = srcd[e];
    }
    out[(size_t)i * it.ldd + j] = (O)v;
  }
}

template <typename DT, typename HT>
__global__ void __launch_bounds__(256) batch_energy_kernel(const BatchItem* items,
                                                           double* __restrict__ part) {
  __shared__ double red[32];
  const BatchItem& it = items[blockIdx.y];
  if ((int)blockIdx.x >= it.gblocks) return;  // the single-solve block layout
  const DT* D = (const DT*)it.D_out;
  const HT* H = (const HT*)it.H;
  double v[1] = {0.0};
  const int warps = blockDim.x / 32;
  const int gw = blockIdx.x * warps + (threadIdx.x >> 5), nw = it.gblocks * warps;
  const int lane = threadIdx.x & 31;
  for (int i = gw; i < it.M; i += nw) {
    for (int j = lane; j < it.M; j += 32)
      v[0] += (double)D[(size_t)i * it.ldd + j] * (double)H[(size_t)i * it.ld + j];
  }
  block_sum<1>(v, red);
  if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = v[0];
}

__global__ void batch_energy_finalize_kernel(const BatchItem* items, int batch,
                                             const double* __restrict__ part, int gstride) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  double e = 0.0;
  for (int k = 0; k < items[b].gblocks; ++k) e += part[(size_t)b * gstride + k];
  items[b].st->E = e;
}
}  // namespace

void launch_batch_control(const double* part, const BatchItem* items, int batch, Ctl ctl,
                          cudaStream_t s) {
  batch_control_kernel<<<batch, kCtlThreads, 0, s>>>(part, items, ctl);
}

void launch_batch_any_active(const BatchItem* items, int batch, unsigned long long cond,
                             int use_cond, int* active_out, cudaStream_t s) {
  batch_any_active_kernel<<<1, 256, 0, s>>>(items, batch, (cudaGraphConditionalHandle)cond,
                                            use_cond, active_out);
}

void launch_batch_check_control(const double* part, const BatchItem* items, int batch, Ctl ctl,
                                cudaStream_t s) {
  batch_check_control_kernel<<<batch, kCtlThreads, 0, s>>>(part, items, ctl);
}

void launch_batch_state_init(const BatchItem* items, int batch, int phase, cudaStream_t s) {
  batch_state_init_kernel<<<(batch + 127) / 128, 128, 0, s>>>(items, batch, phase);
}

void launch_batch_phase_begin(const BatchItem* items, int batch, int phase, cudaStream_t s) {
  batch_phase_begin_kernel<<<(batch + 127) / 128, 128, 0, s>>>(items, batch, phase);
}

// blocks per instance of the batched elementwise kernels
inline int ew_blocks(int maxM) {
  const long long b = ((long long)maxM * maxM + 8191) / 8192;  // ~32 elements a thread
  return (int)(b < 1 ? 1 : (b > 64 ? 64 : b));
}

void launch_batch_x_to_d64(const BatchItem* items, int batch, int maxM, cudaStream_t s) {
  dim3 g(ew_blocks(maxM), batch);
  batch_x_to_d64_kernel<<<g, 256, 0, s>>>(items);
}

void launch_batch_copy_out(const BatchItem* items, int batch, int maxM, int from_x, int out_f64,
                           cudaStream_t s) {
  dim3 g(ew_blocks(maxM), batch);
  if (out_f64)
    batch_copy_out_kernel<double><<<g, 256, 0, s>>>(items, from_x);
  else
    batch_copy_out_kernel<float><<<g, 256, 0, s>>>(items, from_x);
}

void launch_batch_energy(const BatchItem* items, int batch, int out_f64, int h_f64, double* gpart,
                         int gstride, cudaStream_t s) {
  dim3 g(gstride, batch);
  if (out_f64 && h_f64)
    batch_energy_kernel<double, double><<<g, 256, 0, s>>>(items, gpart);
  else if (out_f64)
    batch_energy_kernel<double, float><<<g, 256, 0, s>>>(items, gpart);
  else if (h_f64)
    batch_energy_kernel<float, double><<<g, 256, 0, s>>>(items, gpart);
  else
    batch_energy_kernel<float, float><<<g, 256, 0, s>>>(items, gpart);
  batch_energy_finalize_kernel<<<(batch + 127) / 128, 128, 0, s>>>(items, batch, gpart, gstride);
}
}  // namespace gcp
