// Reverse-mode derivative of the fixed-iteration recursion in FP32 with
// split-FP16 tensor-core products (gcp_backward with GCP_FP32).
//
// The function differentiated is L = <G_D, D_K> + g_E Tr(H D_K) with D_K
// after exactly K steps of Eq. hpcp3 from the guess of Eq. dmguess /
// Eq. pmcpguess (or the HPCP+ or hole guess), as in gcp_adjoint.cu, but every
// iterate lives in the split
// state of the tensor-core path (X = D - theta J in FP32 plus the fp16 halves
// of 2^14 X, Sigma = D^2 - theta^2 J likewise) and c_n follows the rules of
// the fixed-iteration split phase, recorded per step by the control kernel:
//   restoring  c_n = (num + (Tr D - N)/2) / den, the Eq. mcwgamb quotient
//              with the rounding drift of the trace absorbed, so that
//              Tr D_{n+1} = N; dc/dD = ((2D - 3D^2) + J/2 - c (J - 2D)) / den;
//   McWeeny    c_n = 1/2 (Eq. mcweeny3) once ||D^2 - D||_F < 0.05: no dc/dD;
//   identity   the 0/0 guard, or the products have stalled: G passes.
// In exact arithmetic Tr D_n = N and the restoring c_n is Eq. mcwgamb.  The
// adjoint of a restoring step maps G = J to 0 (Tr D_{n+1} = N whatever D_n),
// which holds here to rounding because den and sum G o (S - D) are both taken
// from the same stored iterates.
//
// Forward: the split GEMM1 / control / GEMM2 steps from the guess, keeping X
// every `ckpt` steps and the per-step scalars.  Backward: for each segment,
// last first, the segment's X_n and Sigma_n are recomputed from its
// checkpoint with the same kernels (bit for bit the forward ones); then for
// n from the segment's end down to its start, with D = X + theta J and
// S = Sigma + theta^2 J,
//   P1 = G X,  Q1 = G Sigma,  PT = P1^T + theta G  (= (G D)^T),
//   R1 = X P  (P = G D, given to the product as the rows of PT),
//   G <- (a + b theta - 5 theta^2) G + (b - theta)(P1 + PT)
//        - 2 (Q1 + Q1^T) - (R1 + R1^T) + s dc,
// which is a G + b (P + P^T) - 2 (Q + Q^T + R) + s dc of gcp_adjoint.cu
// with P = G D, Q = G D^2, R = D G D written in the shifted state (G
// symmetric); the three products run on the tensor cores (all tiles: P1, Q1
// and R1 are not symmetric), G and its halves in FP32 with a power-of-two
// scale chosen per step from max |G|, the sum s = 2 sum G o (S - D) and
// den = Tr(D - S) in FP64.  The guess adjoint is the FP64 one of
// gcp_adjoint.cu.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "gcp_device.cuh"
#include "gcp_internal.cuh"

namespace gcp {

namespace {
constexpr int kRed = 256;
constexpr float kXScale = 16384.0f;  // 2^14, the split scale of X and Sigma

__global__ void absmax_kernel(const float* __restrict__ A, size_t n,
                              unsigned int* __restrict__ out) {
  float m = 0.f;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(A[e]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  // non-negative floats order like their bit patterns
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// hi/lo fp16 halves of scale * A (scale a power of two: exact).
// hi/lo fp16 halves of scale * A (scale a power of two: exact); the scale
// from `sptr` when given (a device value, see scale_kernel).
__global__ void split_kernel(const float* __restrict__ A, __half* __restrict__ h,
                             __half* __restrict__ l, size_t n, float scale,
                             const float* __restrict__ sptr) {
  if (sptr) scale = *sptr;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    __half hh, ll;
    Split<false>::split(A[e] * scale, hh, ll);
    h[e] = hh;
    l[e] = ll;
  }
}

// The power of two s = 2^(14 - e) with max |A| < 2^e (amax: the bit pattern
// of max |A|) and 1 / (s xscale), the inverse scale of a product of the
// halves of s A with those of xscale X, into out[0], out[1].
__global__ void scale_kernel(const unsigned int* __restrict__ amax, float xscale,
                             float* __restrict__ out) {
  if (threadIdx.x != 0) return;
  const float m = __uint_as_float(*amax);
  int e = 0;
  frexpf(m > 0.f ? m : 1.f, &e);  // m < 2^e
  const float sc = ldexpf(1.f, 14 - e);
  out[0] = sc;
  out[1] = 1.f / (sc * xscale);
}

// PT = inv P1^T + theta G (32 x 32 tiles through shared memory); P1 is the
// product of the halves, inv (device) its inverse scale.
__global__ void __launch_bounds__(1024) transpose_add_kernel(const float* __restrict__ P1,
                                                             const float* __restrict__ G,
                                                             float* __restrict__ PT, int Mp,
                                                             float theta,
                                                             const float* __restrict__ inv) {
  __shared__ float t[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  const float sc = *inv;
  t[threadIdx.y][threadIdx.x] = P1[(size_t)(by + threadIdx.y) * Mp + bx + threadIdx.x] * sc;
  __syncthreads();
  const int i = bx + threadIdx.y, j = by + threadIdx.x;
  PT[(size_t)i * Mp + j] = t[threadIdx.x][threadIdx.y] + theta * G[(size_t)i * Mp + j];
}

// Per-block partials of sum G o (S - D) and of Tr(S - D), both from the
// same values d = (Sigma - X) + (theta^2 - theta) J (exact in FP64).  The
// step's dc/dD divides by Tr(D - S) taken here rather than by the forward's
// trace partials: then the adjoint maps G = J to J exactly (Tr D_{n+1} =
// Tr D_n for every D, whatever the rounding of the stored iterates), which
// the quotient of two separately rounded near-zero traces would not.
__global__ void __launch_bounds__(256) sdm_reduce_kernel(const float* __restrict__ G,
                                                         const float* __restrict__ Sig,
                                                         const float* __restrict__ X, int M,
                                                         int Mp, double shift,
                                                         double* __restrict__ part) {
  __shared__ double red[64];
  double v[2] = {0.0, 0.0};
  const size_t n = (size_t)Mp * Mp;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / Mp), j = (int)(e % Mp);
    double d = (double)Sig[e] - (double)X[e];
    if (i == j && i < M) {
      d += shift;
      v[1] += d;
    }
    v[0] += (double)G[e] * d;
  }
  block_sum<2>(v, red);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = v[0];
    part[2 * blockIdx.x + 1] = v[1];
  }
}

__global__ void sum_finalize_kernel(const double* __restrict__ part, int nb,
                                    double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int k = 0; k < nb; ++k) {
    a += part[2 * k];
    b += part[2 * k + 1];
  }
  out[0] = a;
  out[1] = b;
}

// G_next from the products (32 x 32 tiles; Q1 and R1 transposed through
// shared memory).  sdm[0] = sum G o (S - D), sdm[1] = Tr(S - D).  restoring:
// c_n = (num + (Tr D - N)/2) / den, whose gradient has the extra J / (2 den);
// otherwise (a McWeeny step, c_n = 1/2) there is no dc/dD term.  The term is
// also dropped when |Tr(D - S)| is at the 0/0 guard den_min.  The padded area
// stays zero.
__global__ void __launch_bounds__(1024) combine_kernel(
    const float* __restrict__ G, const float* __restrict__ P1, const float* __restrict__ PT,
    const float* __restrict__ Q1, const float* __restrict__ R1, const float* __restrict__ X,
    const float* __restrict__ Sig, float* __restrict__ Gn, int M, int Mp, double cg, double cp,
    double theta, double c, int restoring, double den_min, const double* __restrict__ sdm,
    const float* __restrict__ inv_g, const float* __restrict__ inv_r) {
  __shared__ float Qt[32][33];
  __shared__ float Rt[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const float sg = *inv_g, sr = *inv_r;  // inverse scales of P1, Q1 and of R1
  {
    const size_t o = (size_t)(bx + ty) * Mp + by + tx;
    Qt[ty][tx] = Q1[o] * sg;
    Rt[ty][tx] = R1[o] * sr;
  }
  __syncthreads();
  const int i = by + ty, j = bx + tx;
  const size_t o = (size_t)i * Mp + j;
  if (i >= M || j >= M) {
    Gn[o] = 0.f;
    return;
  }
  const double den = -sdm[1];
  const double s = (restoring && fabs(den) > den_min) ? 2.0 * sdm[0] : 0.0;
  const double J = i == j ? 1.0 : 0.0;
  const double d = (double)X[o] + theta * J;
  const double sv = (double)Sig[o] + theta * theta * J;
  const double dc = s != 0.0 ? ((2.0 * d - 3.0 * sv) + 0.5 * J - c * (J - 2.0 * d)) / den : 0.0;
  const double v = cg * (double)G[o] + cp * ((double)(P1[o] * sg) + (double)PT[o]) -
                   2.0 * ((double)(Q1[o] * sg) + (double)Qt[tx][ty]) -
                   ((double)(R1[o] * sr) + (double)Rt[tx][ty]) + s * dc;
  Gn[o] = (float)v;
}

// G = sym(G_D) + g_E H.  D_K is symmetric, so only the symmetric part of
// G_D enters L; the shifted-state update below assumes a symmetric G.  H is
// read from its upper triangle, as everywhere else.
template <typename T>
__global__ void gtc_init_kernel(const T* __restrict__ GD, const T* __restrict__ H, int ld,
                                double gE, int M, int Mp, float* __restrict__ G) {
  const int i = blockIdx.y;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < Mp; j += gridDim.x * blockDim.x) {
    double v = 0.0;
    if (i < M && j < M) {
      v = gE * (double)H[(size_t)(i < j ? i : j) * ld + (i < j ? j : i)];
      if (GD) v += 0.5 * ((double)GD[(size_t)i * ld + j] + (double)GD[(size_t)j * ld + i]);
    }
    G[(size_t)i * Mp + j] = (float)v;
  }
}

// B = sym(A) in FP64: the FP32 combination rounds (i, j) and (j, i)
// differently; the mean is exactly symmetric.
__global__ void to_f64_kernel(const float* __restrict__ A, int Mp, int M, double* __restrict__ B) {
  const int i = blockIdx.y;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x)
    B[(size_t)i * M + j] = 0.5 * ((double)A[(size_t)i * Mp + j] + (double)A[(size_t)j * Mp + i]);
}

inline dim3 rgrid(int cols, int rows) {
  int gx = (cols + 255) / 256;
  if (gx > 8) gx = 8;
  return dim3(gx, rows);
}

struct AdjTcWs {
  int Mp = 0, ck = 0, nck = 0;
  std::vector<void*> bufs;
  // segment slots: X_j and Sigma_j in FP32 and halves, with tensor maps
  std::vector<float*> X, S;
  std::vector<void*> Xh, Xl, Sh, Sl;
  std::vector<TcOperands*> opX, opS;
  float* ckX = nullptr;  // nck checkpoints of X
  float *G = nullptr, *Gn = nullptr, *P1 = nullptr, *Q1 = nullptr, *R1 = nullptr, *PT = nullptr;
  void *Gh = nullptr, *Gl = nullptr, *PTh = nullptr, *PTl = nullptr;
  TcOperands *opG = nullptr, *opPT = nullptr;
  double* G64 = nullptr;  // dL/dD_0 for the guess adjoint (M x M)
  double* DK = nullptr;   // D_K (M x M)
  double* red = nullptr;  // reduction partials and scalars
  unsigned int* amax = nullptr;  // [0]: max |G| bits, [1]: max |PT| bits
  float* scal = nullptr;         // [0] s_G, [1] 1/(s_G 2^14), [2] s_PT, [3] 1/(s_PT 2^14)
  int* kinds = nullptr;  // per-step kStep* of the forward (kcap entries)
  State* rst = nullptr;  // per-step replay states (kcap entries)
  int kcap = 0;
};

void free_ws(AdjTcWs* w) {
  if (w->kinds) cudaFree(w->kinds);
  if (w->rst) cudaFree(w->rst);
  w->kinds = nullptr;
  w->rst = nullptr;
  w->kcap = 0;
  for (void* p : w->bufs) cudaFree(p);
  w->bufs.clear();
  for (TcOperands* o : w->opX) tc_free_operands(o);
  for (TcOperands* o : w->opS) tc_free_operands(o);
  w->opX.clear();
  w->opS.clear();
  if (w->opG) tc_free_operands(w->opG);
  if (w->opPT) tc_free_operands(w->opPT);
  w->opG = w->opPT = nullptr;
  w->X.clear();
  w->S.clear();
  w->Xh.clear();
  w->Xl.clear();
  w->Sh.clear();
  w->Sl.clear();
  w->Mp = w->ck = w->nck = 0;
}

}  // namespace

void adjoint_tc_free(void* ws) {
  AdjTcWs* w = (AdjTcWs*)ws;
  if (!w) return;
  free_ws(w);
  delete w;
}

int adjoint_backward_tc(void** wsp, const void* H, int M, int N, int ld, int h_f64, int guess,
                        const void* GD, double gE, void* dLdH, int K, int ck, State* st,
                        double* part, double* gpart, double* hist, float* scratch,
                        cudaStream_t s, char* err, int errlen) {
#define AT_CK(call)                                                                       \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      snprintf(err, errlen, "gcp_backward (FP32): %s: %s", #call, cudaGetErrorString(e_)); \
      return GCP_ERR_CUDA;                                                                \
    }                                                                                     \
  } while (0)
  AdjTcWs* w = (AdjTcWs*)*wsp;
  if (!w) {
    w = new AdjTcWs;
    *wsp = w;
  }
  if (ck <= 0) ck = 8;
  if (ck > K) ck = K;
  const int Mp = tc_pad(M);
  const size_t n2 = (size_t)Mp * Mp, m2 = (size_t)M * M;
  const int nck = (K - 1) / ck + 1;
  if (w->Mp != Mp || w->ck != ck || w->nck < nck) {
    free_ws(w);
    auto al = [&](size_t bytes) -> void* {
      void* p = nullptr;
      if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
      w->bufs.push_back(p);
      return p;
    };
    bool ok = true;
    // two extra slots beyond the segment: the forward's ping-pong buffers
    for (int j = 0; j < ck + 1 && ok; ++j) {
      float* x = (float*)al(n2 * 4);
      float* sg = (float*)al(n2 * 4);
      void *xh = al(n2 * 2), *xl = al(n2 * 2), *sh = al(n2 * 2), *sl = al(n2 * 2);
      ok = x && sg && xh && xl && sh && sl;
      if (!ok) break;
      w->X.push_back(x);
      w->S.push_back(sg);
      w->Xh.push_back(xh);
      w->Xl.push_back(xl);
      w->Sh.push_back(sh);
      w->Sl.push_back(sl);
      TcOperands *ox = nullptr, *os = nullptr;
      if (tc_make_operands(&ox, xh, xl, Mp, 0, err, errlen) ||
          tc_make_operands(&os, sh, sl, Mp, 0, err, errlen))
        return GCP_ERR_CUDA;
      w->opX.push_back(ox);
      w->opS.push_back(os);
    }
    if (ok) {
      w->ckX = (float*)al((size_t)nck * n2 * 4);
      w->G = (float*)al(n2 * 4);
      w->Gn = (float*)al(n2 * 4);
      w->P1 = (float*)al(n2 * 4);
      w->Q1 = (float*)al(n2 * 4);
      w->R1 = (float*)al(n2 * 4);
      w->PT = (float*)al(n2 * 4);
      w->Gh = al(n2 * 2);
      w->Gl = al(n2 * 2);
      w->PTh = al(n2 * 2);
      w->PTl = al(n2 * 2);
      w->G64 = (double*)al(m2 * 8);
      w->DK = (double*)al(m2 * 8);
      w->red = (double*)al((2 * kRed + 64) * 8);
      w->amax = (unsigned int*)al(64);
      w->scal = (float*)al(64);
      ok = w->ckX && w->G && w->Gn && w->P1 && w->Q1 && w->R1 && w->PT && w->Gh && w->Gl &&
           w->PTh && w->PTl && w->G64 && w->DK && w->red && w->amax && w->scal;
    }
    if (!ok) {
      free_ws(w);
      snprintf(err, errlen, "gcp_backward (FP32): workspace allocation failed");
      return GCP_ERR_CUDA;
    }
    if (tc_make_operands(&w->opG, w->Gh, w->Gl, Mp, 0, err, errlen) ||
        tc_make_operands(&w->opPT, w->PTh, w->PTl, Mp, 0, err, errlen))
      return GCP_ERR_CUDA;
    w->Mp = Mp;
    w->ck = ck;
    w->nck = nck;
  }

  if (w->kcap < K) {
    if (w->kinds) cudaFree(w->kinds);
    if (w->rst) cudaFree(w->rst);
    w->kinds = nullptr;
    w->rst = nullptr;
    w->kcap = 0;
    AT_CK(cudaMalloc((void**)&w->kinds, (size_t)K * sizeof(int)));
    AT_CK(cudaMalloc((void**)&w->rst, (size_t)K * sizeof(State)));
    w->kcap = K;
  }

  // ---------------- forward with checkpoints -----------------------------
  launch_guess_reduce(H, h_f64, M, ld, gpart, s);
  launch_guess_finalize(gpart, guess_partial_blocks(M), M, N, H, h_f64, ld, guess, st, s);
  launch_state_init(st, 1, s);
  // the forward runs in the last two slots (ping-pong), Sigma in slot 0
  const int fa = ck - 1 < 0 ? 0 : ck - 1, fb = ck;
  launch_guess_write_x(H, h_f64, M, ld, w->X[fa], w->Xh[fa], w->Xl[fa], Mp, 0, kXScale, st, s);
  AT_CK(cudaPeekAtLastError());
  State hs;
  AT_CK(cudaMemcpyAsync(&hs, st, sizeof hs, cudaMemcpyDeviceToHost, s));
  AT_CK(cudaStreamSynchronize(s));
  if (hs.no_gap) {
    snprintf(err, errlen, "gcp_backward: H has a zero-width spectrum bound");
    return GCP_ERR_NO_GAP;
  }
  const double theta = hs.theta;
  Ctl ctl{};
  ctl.M = M;
  ctl.N = N;
  ctl.stop = GCP_STOP_IDEMP_FRO;
  ctl.max_iter = K;
  ctl.fixed_iters = K;
  ctl.hist_cap = K + 2;
  ctl.phase = 1;
  ctl.final_phase = 1;
  ctl.endgame = 1;  // the rules of gcp_solve's fixed-iteration split phase
  ctl.tol = 0.0;
  ctl.u = kU32;
  ctl.step_kind = w->kinds;
  AT_CK(cudaMemcpyAsync(w->ckX, w->X[fa], n2 * 4, cudaMemcpyDeviceToDevice, s));
  int cur = fa;
  for (int n = 0; n < K; ++n) {
    const int nxt = cur == fa ? fb : fa;
    int bad = tc_launch_gemm1(w->opX[cur], w->X[cur], w->S[0], w->Sh[0], w->Sl[0], M, Mp,
                              nullptr, 1, M, part, st, 0, kXScale, scratch, s);
    launch_control(part, tc_num_tiles(Mp), st, hist, ctl, 0ull, 0, s);
    bad = bad || tc_launch_gemm2(w->opS[0], w->opX[cur], w->X[cur], w->S[0], w->X[nxt],
                                 w->Xh[nxt], w->Xl[nxt], M, Mp, st, 0, kXScale, scratch, s);
    if (bad) {
      snprintf(err, errlen, "gcp_backward (FP32): forward launch failed: %s",
               cudaGetErrorString(cudaGetLastError()));
      return GCP_ERR_CUDA;
    }
    cur = nxt;
    if ((n + 1) % ck == 0 && n + 1 < K)
      AT_CK(cudaMemcpyAsync(w->ckX + (size_t)((n + 1) / ck) * n2, w->X[cur], n2 * 4,
                            cudaMemcpyDeviceToDevice, s));
  }
  AT_CK(cudaPeekAtLastError());
  // D_K = X_K + theta J in FP64 (the g_E D_K term of dL/dH)
  launch_copy_out_x(w->X[cur], w->X[cur], st, M, Mp, w->DK, 1, M, s);
  std::vector<double> rec((size_t)(K + 2) * GCP_HISTORY_FIELDS);
  AT_CK(cudaMemcpyAsync(&hs, st, sizeof hs, cudaMemcpyDeviceToHost, s));
  AT_CK(cudaStreamSynchronize(s));
  if (hs.timeout) {
    snprintf(err, errlen, "gcp_backward (FP32): a device-side wait gave up");
    return GCP_ERR_TIMEOUT;
  }
  const int nrec = hs.hist_n < K ? hs.hist_n : K;
  if (nrec > 0)
    AT_CK(cudaMemcpy(rec.data(), hist, (size_t)nrec * GCP_HISTORY_FIELDS * sizeof(double),
                     cudaMemcpyDeviceToHost));
  if (nrec < K) {
    snprintf(err, errlen, "gcp_backward (FP32): forward recorded %d of %d steps", nrec, K);
    return GCP_ERR_CUDA;
  }
  std::vector<int> kind(K);
  AT_CK(cudaMemcpy(kind.data(), w->kinds, (size_t)K * sizeof(int), cudaMemcpyDeviceToHost));

  // ---------------- backward ---------------------------------------------
  if (h_f64)
    gtc_init_kernel<double><<<rgrid(Mp, Mp), 256, 0, s>>>((const double*)GD, (const double*)H, ld,
                                                          gE, M, Mp, w->G);
  else
    gtc_init_kernel<float><<<rgrid(Mp, Mp), 256, 0, s>>>((const float*)GD, (const float*)H, ld,
                                                         gE, M, Mp, w->G);
  // One replay state per step, uploaded once: the recomputed steps read
  // their coefficients from it, and every kernel of step n that may raise a
  // timeout writes it there, so the backward pass needs no host round trip
  // until its end.
  std::vector<State> rs((size_t)K);
  for (int n = 0; n < K; ++n) {
    State& r = rs[(size_t)n];
    memset(&r, 0, sizeof r);
    const double c = rec[(size_t)n * GCP_HISTORY_FIELDS + 5];
    const bool applied = kind[n] != kStepIdentity;
    r.theta = theta;
    r.apply = applied ? 1 : 0;
    r.a = applied ? 1.0 - 2.0 * c : 1.0;
    r.b = applied ? 2.0 + 2.0 * c : 0.0;
    r.g3 = -2.0;  // HPCP (Eq. hpcp3)
    r.xshift = applied ? 2.0 * theta * (1.0 - theta) * (theta - c) : 0.0;
  }
  AT_CK(cudaMemcpyAsync(w->rst, rs.data(), (size_t)K * sizeof(State), cudaMemcpyHostToDevice, s));
  const dim3 tg(Mp / 32, Mp / 32), tb(32, 32);
  // the forward's 0/0 guard of the split phase
  const double den_min = 16.0 * sqrt((double)M) * kU32;
  const int eb = (int)((n2 + 255) / 256 < 1184 ? (n2 + 255) / 256 : 1184);
  for (int seg = (K - 1) / ck; seg >= 0; --seg) {
    const int n0 = seg * ck, n1 = (n0 + ck < K) ? n0 + ck : K;
    AT_CK(cudaMemcpyAsync(w->X[0], w->ckX + (size_t)seg * n2, n2 * 4, cudaMemcpyDeviceToDevice, s));
    split_kernel<<<eb, 256, 0, s>>>(w->X[0], (__half*)w->Xh[0], (__half*)w->Xl[0], n2, kXScale,
                                    nullptr);
    for (int n = n0; n < n1; ++n) {
      const int j = n - n0;
      State* sn = w->rst + n;
      if (tc_launch_gemm1(w->opX[j], w->X[j], w->S[j], w->Sh[j], w->Sl[j], M, Mp, nullptr, 1, M,
                          part, sn, 0, kXScale, scratch, s) ||
          (n + 1 < n1 && tc_launch_gemm2(w->opS[j], w->opX[j], w->X[j], w->S[j], w->X[j + 1],
                                         w->Xh[j + 1], w->Xl[j + 1], M, Mp, sn, 0, kXScale,
                                         scratch, s))) {
        snprintf(err, errlen, "gcp_backward (FP32): recompute launch failed: %s",
                 cudaGetErrorString(cudaGetLastError()));
        return GCP_ERR_CUDA;
      }
    }
    for (int n = n1 - 1; n >= n0; --n) {
      const int j = n - n0;
      State* sn = w->rst + n;
      const double* Rc = rec.data() + (size_t)n * GCP_HISTORY_FIELDS;
      const double c = Rc[5];
      if (kind[n] == kStepIdentity) continue;  // G passes through
      const double a = 1.0 - 2.0 * c, b = 2.0 + 2.0 * c;
      // s/2 = sum G o (S - D) and Tr(S - D) (McWeeny steps: c is constant)
      if (kind[n] == kStepRestoring) {
        sdm_reduce_kernel<<<kRed, 256, 0, s>>>(w->G, w->S[j], w->X[j], M, Mp,
                                               theta * theta - theta, w->red);
        sum_finalize_kernel<<<1, 32, 0, s>>>(w->red, kRed, w->red + 2 * kRed);
      }
      // halves of G and of PT at power-of-two scales that keep their
      // entries below 2^14 (scale_kernel); the products are stored unscaled
      // and the kernels that read them apply the inverse scales
      AT_CK(cudaMemsetAsync(w->amax, 0, 8, s));
      absmax_kernel<<<eb, 256, 0, s>>>(w->G, n2, w->amax);
      scale_kernel<<<1, 32, 0, s>>>(w->amax, kXScale, w->scal);
      split_kernel<<<eb, 256, 0, s>>>(w->G, (__half*)w->Gh, (__half*)w->Gl, n2, 1.f, w->scal);
      if (tc_launch_product(w->opG, w->opX[j], w->P1, Mp, 0, 1.f, sn, scratch, s) ||
          tc_launch_product(w->opG, w->opS[j], w->Q1, Mp, 0, 1.f, sn, scratch, s)) {
        snprintf(err, errlen, "gcp_backward (FP32): product launch failed: %s",
                 cudaGetErrorString(cudaGetLastError()));
        return GCP_ERR_CUDA;
      }
      transpose_add_kernel<<<tg, tb, 0, s>>>(w->P1, w->G, w->PT, Mp, (float)theta, w->scal + 1);
      absmax_kernel<<<eb, 256, 0, s>>>(w->PT, n2, w->amax + 1);
      scale_kernel<<<1, 32, 0, s>>>(w->amax + 1, kXScale, w->scal + 2);
      split_kernel<<<eb, 256, 0, s>>>(w->PT, (__half*)w->PTh, (__half*)w->PTl, n2, 1.f,
                                      w->scal + 2);
      if (tc_launch_product(w->opX[j], w->opPT, w->R1, Mp, 0, 1.f, sn, scratch, s)) {
        snprintf(err, errlen, "gcp_backward (FP32): product launch failed: %s",
                 cudaGetErrorString(cudaGetLastError()));
        return GCP_ERR_CUDA;
      }
      combine_kernel<<<tg, tb, 0, s>>>(w->G, w->P1, w->PT, w->Q1, w->R1, w->X[j], w->S[j], w->Gn,
                                       M, Mp, a + b * theta - 5.0 * theta * theta, b - theta,
                                       theta, c, kind[n] == kStepRestoring ? 1 : 0, den_min,
                                       w->red + 2 * kRed, w->scal + 1, w->scal + 3);
      AT_CK(cudaPeekAtLastError());
      float* t = w->G;
      w->G = w->Gn;
      w->Gn = t;
    }
  }
  // any wait of the recomputation or of the products that gave up
  AT_CK(cudaMemcpyAsync(rs.data(), w->rst, (size_t)K * sizeof(State), cudaMemcpyDeviceToHost, s));
  AT_CK(cudaStreamSynchronize(s));
  for (int n = 0; n < K; ++n)
    if (rs[(size_t)n].timeout) {
      snprintf(err, errlen, "gcp_backward (FP32): a device-side wait gave up");
      return GCP_ERR_TIMEOUT;
    }
  // ---------------- guess (FP64, shared with gcp_adjoint.cu) ---------------
  to_f64_kernel<<<rgrid(M, M), 256, 0, s>>>(w->G, Mp, M, w->G64);
  AT_CK(cudaPeekAtLastError());
  return adjoint_guess(H, M, N, ld, h_f64, guess, w->G64, w->DK, gE, dLdH, gpart, st, s, err,
                       errlen);
#undef AT_CK
}

}  // namespace gcp
