// Reverse-mode derivative of the fixed-iteration recursion (gcp_backward).
//
// L = <G_D, D_K> + g_E Tr(H D_K), D_K after exactly K steps of Eq. hpcp3
// (or of the PM step of Eq. pm1) from the canonical, HPCP+ or hole guess.
// FP64 throughout.
//
// Forward: the FP64 step kernels from the guess, keeping D every `ckpt`
// steps and the per-step scalars (c_n, Tr D_n, Tr D_n^2).  Backward: for each
// segment, last first, the iterates D_n and S_n = D_n^2 are recomputed from
// its checkpoint with the same kernels (so they equal the forward ones bit
// for bit), then for n from the segment's end down to its start, for
// D+ = a D + b D^2 + g3 D^3 (HPCP: a = 1 - 2c, b = 2 + 2c, g3 = -2; PMCP:
// the coefficients of Eq. pm1 on the branch c took),
//   G <- a G + b (P + P^T) + g3 (Q + Q^T + R) + s dc
//   P = G D, Q = G S (= G D^2), R = D P (= D G D),
//   s = dL/dc = sum G o (a' D + b' S) + g3' sum Q o D  (' = d/dc),
//   dc = dc/dD = [(2D - 3S) - c (I - 2D)] / (Tr D - Tr S).
// A step past the 0/0 guard was an identity step and passes G through.
// Last, the guess D_0 = theta I + b (mu I - H): with G_0 = dL/dD_0,
//   dL/dH = -b G_0 + (g_mu / M) I + sum over the Gershgorin branches that
//           set b of w_k g_ext,k * (row of their extreme disc, symmetrised)
//           [+ g_b b (mu I - H) / F for HPCP+ with an interior alpha]
//           + g_E D_K,
// g_b = sum G_0 o (mu I - H), g_mu = b Tr G_0 + sum_k w_k (db_k/dmu) g_b,
// g_ext,k = (db_k/dH_ext) g_b.  b is beta_min (canonical: weight 1 on the
// smaller bound), beta_max (hole), or for HPCP+ (Eq. hpcpguess)
// alpha beta_min + (1 - alpha) beta_max: with alpha fixed (1/2 for the
// middle fillings, or clamped) the weights alpha, 1 - alpha; with alpha
// the root of Eq. hpcpguessalpha, b^2 = (target - M theta^2) / F,
// F = ||mu I - H||_F^2, so db/dH = b (mu I - H) / F.  The row of the
// extreme disc i* carries sign(H_{i* j}) (a subgradient where H_{i*j} = 0)
// and 1 on its diagonal.
#include <stdio.h>
#include <string.h>

#include <vector>

#include "gcp_device.cuh"
#include "gcp_fp64_tile.cuh"
#include "gcp_internal.cuh"

namespace gcp {

// Coefficients of D+ = a D + b D^2 + g3 D^3 for c and the method, and their
// c-derivatives: the expressions of set_coeffs (gcp_control.cu), so that the
// replayed steps equal the forward ones bit for bit.
StepCoeffs step_coeffs(double c, int method) {
  StepCoeffs k;
  if (method == GCP_METHOD_PMCP) {
    if (c <= 0.5) {
      const double q = 1.0 - c;
      k.a = (1.0 - 2.0 * c) / q;
      k.b = (1.0 + c) / q;
      k.g3 = -1.0 / q;
      k.da = -1.0 / (q * q);
      k.db = 2.0 / (q * q);
      k.dg3 = -1.0 / (q * q);
    } else {
      k.a = 0.0;
      k.b = (1.0 + c) / c;
      k.g3 = -1.0 / c;
      k.da = 0.0;
      k.db = -1.0 / (c * c);
      k.dg3 = 1.0 / (c * c);
    }
  } else {
    k.a = 1.0 - 2.0 * c;
    k.b = 2.0 + 2.0 * c;
    k.g3 = -2.0;
    k.da = -2.0;
    k.db = 2.0;
    k.dg3 = 0.0;
  }
  return k;
}

namespace {
constexpr int kBT = 32;
constexpr int kRedBlocks = 256;

// C = A B over BT x BT tiles; A symmetric.  upper: only tiles on or above
// the diagonal, elements above the diagonal mirrored (C symmetric).
__global__ void __launch_bounds__(kF64Threads) adj_gemm_kernel(const double* __restrict__ A,
                                                               const double* __restrict__ B,
                                                               double* __restrict__ C, int M,
                                                               int upper) {
  __shared__ double As[kF64BK][kBT];
  __shared__ double Bs[kF64BK][kBT];
  constexpr int RT = kBT / 16;
  const int T = (M + kBT - 1) / kBT;
  int bi, bj;
  if (upper) {
    f64_tile_coords(blockIdx.x, T, bi, bj);
  } else {
    bi = blockIdx.x / T;
    bj = blockIdx.x % T;
  }
  const int m0 = bi * kBT, n0 = bj * kBT;
  double acc[RT][RT];
  f64_mainloop<kBT>(A, B, M, M, m0, n0, acc, As, Bs);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < RT; ++i) {
    const int r = m0 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < RT; ++j) {
      const int c = n0 + tx + 16 * j;
      if (r >= M || c >= M) continue;
      if (upper) {
        if (c < r) continue;
        C[(size_t)r * M + c] = acc[i][j];
        if (c != r) C[(size_t)c * M + r] = acc[i][j];
      } else {
        C[(size_t)r * M + c] = acc[i][j];
      }
    }
  }
}

// Per-block partial sums of up to three elementwise products (FP64):
// v0 = sum X0 o (Y0 - Z0), v1 = sum diag(X1), v2 = sum X1 o W (W in any dtype).
template <typename WT>
__global__ void __launch_bounds__(256) adj_reduce_kernel(const double* __restrict__ X0,
                                                         const double* __restrict__ Y0,
                                                         const double* __restrict__ Z0,
                                                         const double* __restrict__ X1,
                                                         const WT* __restrict__ W, int ldw, int M,
                                                         double* __restrict__ part) {
  __shared__ double red[32 * 3];
  double v[3] = {0.0, 0.0, 0.0};
  const size_t n = (size_t)M * M;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / M), j = (int)(e % M);
    if (X0) v[0] += X0[e] * (Y0[e] - Z0[e]);
    if (X1) {
      if (i == j) v[1] += X1[e];
      if (W) v[2] += X1[e] * (double)W[(size_t)i * ldw + j];
    }
  }
  block_sum<3>(v, red);
  if (threadIdx.x == 0) {
    part[blockIdx.x * 3 + 0] = v[0];
    part[blockIdx.x * 3 + 1] = v[1];
    part[blockIdx.x * 3 + 2] = v[2];
  }
}

__global__ void adj_reduce_finalize_kernel(const double* __restrict__ part, int nb,
                                           double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double a = 0.0, b = 0.0, c = 0.0;
  for (int k = 0; k < nb; ++k) {
    a += part[k * 3 + 0];
    b += part[k * 3 + 1];
    c += part[k * 3 + 2];
  }
  out[0] = a;
  out[1] = b;
  out[2] = c;
}

// Per-block partials of sum G o (da D + db S) and sum Q o D (the dL/dc of a
// step), the first as one elementwise product.
__global__ void __launch_bounds__(256) adj_s_reduce_kernel(const double* __restrict__ G,
                                                           const double* __restrict__ D,
                                                           const double* __restrict__ S,
                                                           const double* __restrict__ Q,
                                                           double da, double db, int M,
                                                           double* __restrict__ part) {
  __shared__ double red[32 * 3];
  double v[3] = {0.0, 0.0, 0.0};
  const size_t n = (size_t)M * M;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    v[0] += G[e] * (da * D[e] + db * S[e]);
    if (Q) v[1] += Q[e] * D[e];
  }
  block_sum<3>(v, red);
  if (threadIdx.x == 0) {
    part[blockIdx.x * 3 + 0] = v[0];
    part[blockIdx.x * 3 + 1] = v[1];
    part[blockIdx.x * 3 + 2] = 0.0;
  }
}

// G_next = a G + b (P + P^T) + g3 (Q + Q^T + R) + s dc, s = sred[0] +
// dg3 sred[1]; 32 x 32 tiles with the transposed tiles of P and Q staged in
// shared memory.
__global__ void __launch_bounds__(1024) adj_combine_kernel(
    const double* __restrict__ G, const double* __restrict__ P, const double* __restrict__ Q,
    const double* __restrict__ R, const double* __restrict__ D, const double* __restrict__ S,
    double* __restrict__ Gn, int M, double a, double b, double g3, double dg3, double c,
    double den, const double* __restrict__ sred) {
  __shared__ double Pt[32][33];
  __shared__ double Qt[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  // transposed tile: rows bx.., columns by..
  {
    const int r = bx + ty, cc = by + tx;
    const bool in = r < M && cc < M;
    Pt[ty][tx] = in ? P[(size_t)r * M + cc] : 0.0;
    Qt[ty][tx] = in ? Q[(size_t)r * M + cc] : 0.0;
  }
  __syncthreads();
  const int i = by + ty, j = bx + tx;
  if (i >= M || j >= M) return;
  const size_t o = (size_t)i * M + j;
  const double s = dg3 != 0.0 ? sred[0] + dg3 * sred[1] : sred[0];
  const double pji = Pt[tx][ty], qji = Qt[tx][ty];
  const double d = D[o], sv = S[o];
  const double dc = ((2.0 * d - 3.0 * sv) - c * ((i == j ? 1.0 : 0.0) - 2.0 * d)) / den;
  Gn[o] = a * G[o] + b * (P[o] + pji) + g3 * (Q[o] + qji + R[o]) + s * dc;
}

template <typename T>
__global__ void adj_init_kernel(const T* __restrict__ GD, const T* __restrict__ H, int ld,
                                double gE, int M, double* __restrict__ G) {
  const int i = blockIdx.y;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
    double v = gE * (double)H[(size_t)i * ld + j];
    if (GD) v += (double)GD[(size_t)i * ld + j];
    G[(size_t)i * M + j] = v;
  }
}

// Gershgorin extreme discs: per block (max of H_ii + r_i, its row) and
// (min of H_ii - r_i, its row); ties keep the smallest row.
template <typename T>
__global__ void __launch_bounds__(256) adj_gersh_kernel(const T* __restrict__ H, int ld, int M,
                                                        double* __restrict__ part) {
  __shared__ double sv[8][2];
  __shared__ int si[8][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gw = blockIdx.x * 8 + warp, nw = gridDim.x * 8;
  double hv = -INFINITY, lv = INFINITY;
  int hi = M, li = M;
  for (int i = gw; i < M; i += nw) {
    const T* row = H + (size_t)i * ld;
    double r = 0.0;
    for (int j = lane; j < M; j += 32) r += fabs((double)row[j]);
    r = warp_sum(r);
    const double d = (double)row[i];
    r -= fabs(d);
    if (d + r > hv) {
      hv = d + r;
      hi = i;
    }
    if (d - r < lv) {
      lv = d - r;
      li = i;
    }
  }
  if (lane == 0) {
    sv[warp][0] = hv;
    si[warp][0] = hi;
    sv[warp][1] = lv;
    si[warp][1] = li;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) {
      if (sv[w][0] > sv[0][0] || (sv[w][0] == sv[0][0] && si[w][0] < si[0][0])) {
        sv[0][0] = sv[w][0];
        si[0][0] = si[w][0];
      }
      if (sv[w][1] < sv[0][1] || (sv[w][1] == sv[0][1] && si[w][1] < si[0][1])) {
        sv[0][1] = sv[w][1];
        si[0][1] = si[w][1];
      }
    }
    part[blockIdx.x * 4 + 0] = sv[0][0];
    part[blockIdx.x * 4 + 1] = (double)si[0][0];
    part[blockIdx.x * 4 + 2] = sv[0][1];
    part[blockIdx.x * 4 + 3] = (double)si[0][1];
  }
}

__global__ void adj_gersh_finalize_kernel(const double* __restrict__ part, int nb,
                                          double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double hv = -INFINITY, lv = INFINITY, hi = 1e300, li = 1e300;
  for (int k = 0; k < nb; ++k) {
    const double* p = part + k * 4;
    if (p[0] > hv || (p[0] == hv && p[1] < hi)) {
      hv = p[0];
      hi = p[1];
    }
    if (p[2] < lv || (p[2] == lv && p[3] < li)) {
      lv = p[2];
      li = p[3];
    }
  }
  out[0] = hi;
  out[1] = li;
}

__device__ __forceinline__ double sgn(double x) { return (double)((x > 0.0) - (x < 0.0)); }

// ||mu I - H||_F^2 per block (mu from the state), for the HPCP+ guess.
template <typename T>
__global__ void __launch_bounds__(256) adj_frob_kernel(const T* __restrict__ H, int ld, int M,
                                                       const State* __restrict__ st,
                                                       double* __restrict__ part) {
  __shared__ double red[32];
  const double mu = st->mu;
  double v[1] = {0.0};
  const size_t n = (size_t)M * M;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / M), j = (int)(e % M);
    const double x = (i == j ? mu : 0.0) - (double)H[(size_t)i * ld + j];
    v[0] += x * x;
  }
  block_sum<1>(v, red);
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
}

__global__ void adj_sum_kernel(const double* __restrict__ part, int nb, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double a = 0.0;
  for (int k = 0; k < nb; ++k) a += part[k];
  *out = a;
}

// dL/dH = sym(-b G0 + (g_mu/M) I + sum_k w_k g_ext,k row(i*_k) [+ sqrt
// term]) + g_E D_K (see the header comment).  sc: [0] i*_max, [1] i*_min
// (from the Gershgorin pass), [3] Tr G0, [4] sum G0 o H, [5] F.
template <typename T>
__global__ void adj_guess_kernel(const double* __restrict__ G0, const T* __restrict__ H, int ld,
                                 int M, int N, int mode, const State* __restrict__ st,
                                 const double* __restrict__ sc, const double* __restrict__ DK,
                                 double gE, T* __restrict__ out) {
  const double theta = st->theta, mu = st->mu, b = st->beta2, alpha = st->alpha;
  const double hmin = st->hmin, hmax = st->hmax;
  const double trG = sc[3], gH = sc[4], F = sc[5];
  const double g_b = mu * trG - gH;  // sum G0 o (mu I - H)
  double g_mu = b * trG;
  const double b_up = hmax - mu > 0.0 ? theta / (hmax - mu) : INFINITY;
  const double b_lo = mu - hmin > 0.0 ? (1.0 - theta) / (mu - hmin) : INFINITY;
  const bool up_min = b_up <= b_lo;
  // weights of the smaller and the larger bound in b, and the sqrt form
  double w_min = 1.0, w_max = 0.0, c_sq = 0.0;
  if (isfinite(fmax(b_up, b_lo))) {
    if (mode == GCP_GUESS_HOLE) {
      w_min = 0.0;
      w_max = 1.0;
    } else if (mode == GCP_GUESS_HPCP_PLUS) {
      const double delta = 2.0 / 3.0;
      const bool has_target = theta <= 1.0 - delta || theta >= delta;
      if (has_target && alpha > 0.0 && alpha < 1.0 && F > 0.0) {
        w_min = w_max = 0.0;
        c_sq = g_b * b / F;
      } else {
        w_min = alpha;
        w_max = 1.0 - alpha;
      }
    }
  }
  const double w_up = up_min ? w_min : w_max, w_lo = up_min ? w_max : w_min;
  double g_up = 0.0, g_lo = 0.0;
  if (w_up != 0.0) {
    const double w = theta / ((hmax - mu) * (hmax - mu));
    g_mu += w_up * g_b * w;
    g_up = -w_up * g_b * w;
  }
  if (w_lo != 0.0) {
    const double w = (1.0 - theta) / ((mu - hmin) * (mu - hmin));
    g_mu -= w_lo * g_b * w;
    g_lo = w_lo * g_b * w;
  }
  const int iu = (int)sc[0], il = (int)sc[1];
  const int i = blockIdx.y;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
    double v = -b * G0[(size_t)i * M + j];
    if (i == j) v += g_mu / (double)M;
    // rows of the extreme discs, symmetrised over (i, j) and (j, i)
    if (g_up != 0.0) {
      double row = 0.0;
      if (i == iu) row += (j == iu) ? 1.0 : sgn((double)H[(size_t)iu * ld + j]);
      if (j == iu) row += (i == iu) ? 1.0 : sgn((double)H[(size_t)iu * ld + i]);
      v += 0.5 * g_up * row;
    }
    if (g_lo != 0.0) {
      double row = 0.0;
      if (i == il) row += (j == il) ? 1.0 : -sgn((double)H[(size_t)il * ld + j]);
      if (j == il) row += (i == il) ? 1.0 : -sgn((double)H[(size_t)il * ld + i]);
      v += 0.5 * g_lo * row;
    }
    if (c_sq != 0.0) {
      const double hs = 0.5 * ((double)H[(size_t)i * ld + j] + (double)H[(size_t)j * ld + i]);
      v += c_sq * ((i == j ? mu : 0.0) - hs);
    }
    v += gE * DK[(size_t)i * M + j];
    out[(size_t)i * ld + j] = (T)v;
  }
}

inline dim3 row_grid(int M) {
  int gx = (M + 255) / 256;
  if (gx > 8) gx = 8;
  return dim3(gx, M);
}

struct AdjWs {
  int M = 0, K = 0, ck = 0;
  double* base = nullptr;
  size_t bytes = 0;
};

double* g_guess_tmp = nullptr;  // per-process scratch of adjoint_guess (device)

}  // namespace

// dL/dH from G0 = dL/dD_0 (FP64, M x M): the guess adjoint of Eq. dmguess /
// Eq. pmcpguess (see the header comment) plus g_E D_K.
int adjoint_guess(const void* H, int M, int N, int ld, int h_f64, int guess, const double* G0,
                  const double* DK, double gE, void* dLdH, double* gpart, State* st,
                  cudaStream_t s, char* err, int errlen) {
#define AG_CK(call)                                                                  \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      snprintf(err, errlen, "gcp_backward: %s: %s", #call, cudaGetErrorString(e_));  \
      return GCP_ERR_CUDA;                                                           \
    }                                                                                \
  } while (0)
  if (!g_guess_tmp) AG_CK(cudaMalloc((void**)&g_guess_tmp, (3 * kRedBlocks + 64) * sizeof(double)));
  double* rpart = g_guess_tmp;
  double* sc = g_guess_tmp + 3 * kRedBlocks;
  // restore the guess parameters (a replay state may have overwritten them)
  launch_guess_reduce(H, h_f64, M, ld, gpart, s);
  launch_guess_finalize(gpart, guess_partial_blocks(M), M, N, H, h_f64, ld, guess, st, s);
  if (h_f64) {
    adj_gersh_kernel<double><<<kRedBlocks, 256, 0, s>>>((const double*)H, ld, M, rpart);
    adj_gersh_finalize_kernel<<<1, 32, 0, s>>>(rpart, kRedBlocks, sc);
    adj_reduce_kernel<double><<<kRedBlocks, 256, 0, s>>>(nullptr, nullptr, nullptr, G0,
                                                        (const double*)H, ld, M, rpart);
  } else {
    adj_gersh_kernel<float><<<kRedBlocks, 256, 0, s>>>((const float*)H, ld, M, rpart);
    adj_gersh_finalize_kernel<<<1, 32, 0, s>>>(rpart, kRedBlocks, sc);
    adj_reduce_kernel<float><<<kRedBlocks, 256, 0, s>>>(nullptr, nullptr, nullptr, G0,
                                                       (const float*)H, ld, M, rpart);
  }
  adj_reduce_finalize_kernel<<<1, 32, 0, s>>>(rpart, kRedBlocks, sc + 2);
  if (guess == GCP_GUESS_HPCP_PLUS) {  // F = ||mu I - H||_F^2 into sc[5]
    if (h_f64)
      adj_frob_kernel<double><<<kRedBlocks, 256, 0, s>>>((const double*)H, ld, M, st, rpart);
    else
      adj_frob_kernel<float><<<kRedBlocks, 256, 0, s>>>((const float*)H, ld, M, st, rpart);
    adj_sum_kernel<<<1, 32, 0, s>>>(rpart, kRedBlocks, sc + 5);
  } else {
    AG_CK(cudaMemsetAsync(sc + 5, 0, sizeof(double), s));
  }
  if (h_f64)
    adj_guess_kernel<double><<<row_grid(M), 256, 0, s>>>(G0, (const double*)H, ld, M, N, guess, st,
                                                        sc, DK, gE, (double*)dLdH);
  else
    adj_guess_kernel<float><<<row_grid(M), 256, 0, s>>>(G0, (const float*)H, ld, M, N, guess, st,
                                                       sc, DK, gE, (float*)dLdH);
  AG_CK(cudaPeekAtLastError());
  AG_CK(cudaStreamSynchronize(s));
#undef AG_CK
  return GCP_OK;
}

void adjoint_free(void* ws) {
  AdjWs* w = (AdjWs*)ws;
  if (!w) return;
  cudaFree(w->base);
  delete w;
}

// The backward pass; `*ws` is the caller's workspace cache (grown here).
// D64/S64/part/st/hist: the handle's FP64 buffers (>= M x M), tile partials,
// solver state and a history buffer of at least K + 2 records.
int adjoint_backward(void** wsp, const void* H, int M, int N, int ld, int h_f64, int guess,
                     int method, const void* GD, double gE, void* dLdH, int K, int ck,
                     double* D64_0, double* D64_1, double* S64, double* part, double* gpart,
                     State* st, double* hist, cudaStream_t s, char* err, int errlen) {
#define AD_CK(call)                                                                  \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      snprintf(err, errlen, "gcp_backward: %s: %s", #call, cudaGetErrorString(e_));  \
      return GCP_ERR_CUDA;                                                           \
    }                                                                                \
  } while (0)
  AdjWs* w = (AdjWs*)*wsp;
  if (!w) {
    w = new AdjWs;
    *wsp = w;
  }
  if (ck <= 0) ck = 8;
  if (ck > K) ck = K;
  const size_t m2 = (size_t)M * M;
  const int nck = (K - 1) / ck + 1;  // checkpoints D_0, D_ck, ...
  // checkpoints, segment D and S, G, Gn, P, Q, R, D_K, scalars
  const size_t need = ((size_t)nck + 2 * (size_t)ck + 6) * m2 + 4096 + 3 * kRedBlocks + 64;
  if (need * sizeof(double) > w->bytes) {
    cudaFree(w->base);
    w->base = nullptr;
    w->bytes = 0;
    AD_CK(cudaMalloc((void**)&w->base, need * sizeof(double)));
    w->bytes = need * sizeof(double);
  }
  double* p = w->base;
  double* ckpt = p;
  p += (size_t)nck * m2;
  double* segD = p;
  p += (size_t)ck * m2;
  double* segS = p;
  p += (size_t)ck * m2;
  double* G = p;
  p += m2;
  double* Gn = p;
  p += m2;
  double* P = p;
  p += m2;
  double* Q = p;
  p += m2;
  double* R = p;
  p += m2;
  double* DK = p;
  p += m2;
  double* rpart = p;
  p += 3 * kRedBlocks;
  double* sc = p;  // scalars

  // ---------------- forward with checkpoints -----------------------------
  launch_guess_reduce(H, h_f64, M, ld, gpart, s);
  launch_guess_finalize(gpart, guess_partial_blocks(M), M, N, H, h_f64, ld, guess, st, s);
  launch_state_init(st, 0, s);
  launch_guess_write_d(H, h_f64, M, ld, D64_0, 1, M, M, st, s);
  AD_CK(cudaPeekAtLastError());
  State hs;
  AD_CK(cudaMemcpyAsync(&hs, st, sizeof hs, cudaMemcpyDeviceToHost, s));
  AD_CK(cudaStreamSynchronize(s));
  if (hs.no_gap) {
    snprintf(err, errlen, "gcp_backward: H has a zero-width spectrum bound");
    return GCP_ERR_NO_GAP;
  }
  Ctl ctl{};
  ctl.M = M;
  ctl.N = N;
  ctl.stop = GCP_STOP_IDEMP_FRO;
  ctl.max_iter = K;
  ctl.fixed_iters = K;
  ctl.hist_cap = K + 2;
  ctl.phase = 0;
  ctl.final_phase = 1;
  ctl.endgame = 0;
  ctl.tol = 0.0;
  ctl.u = kU64;
  ctl.method = method;
  double* buf[2] = {D64_0, D64_1};
  AD_CK(cudaMemcpyAsync(ckpt, D64_0, m2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  for (int n = 0; n < K; ++n) {
    launch_f64_gemm1(buf[n & 1], S64, M, M, nullptr, 1, M, part, st, s);
    launch_control(part, f64_num_tiles(M), st, hist, ctl, 0ull, 0, s);
    launch_f64_gemm2(S64, buf[n & 1], buf[(n & 1) ^ 1], M, M, st, s);
    if ((n + 1) % ck == 0 && n + 1 < K)
      AD_CK(cudaMemcpyAsync(ckpt + (size_t)((n + 1) / ck) * m2, buf[(n + 1) & 1],
                            m2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  AD_CK(cudaPeekAtLastError());
  AD_CK(cudaMemcpyAsync(DK, buf[K & 1], m2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  std::vector<double> rec((size_t)(K + 2) * GCP_HISTORY_FIELDS);
  AD_CK(cudaMemcpyAsync(&hs, st, sizeof hs, cudaMemcpyDeviceToHost, s));
  AD_CK(cudaStreamSynchronize(s));
  const int nrec = hs.hist_n < K ? hs.hist_n : K;
  if (nrec > 0)
    AD_CK(cudaMemcpy(rec.data(), hist, (size_t)nrec * GCP_HISTORY_FIELDS * sizeof(double),
                     cudaMemcpyDeviceToHost));
  if (nrec < K) {
    snprintf(err, errlen, "gcp_backward: forward recorded %d of %d steps", nrec, K);
    return GCP_ERR_CUDA;
  }

  // ---------------- backward ---------------------------------------------
  if (h_f64)
    adj_init_kernel<double><<<row_grid(M), 256, 0, s>>>((const double*)GD, (const double*)H, ld,
                                                       gE, M, G);
  else
    adj_init_kernel<float><<<row_grid(M), 256, 0, s>>>((const float*)GD, (const float*)H, ld, gE,
                                                      M, G);
  const int T = (M + kBT - 1) / kBT;
  const int nfull = T * T, nup = T * (T + 1) / 2;
  State rs;  // replay state for the recomputation (apply, a, b, g3)
  memset(&rs, 0, sizeof rs);
  for (int seg = (K - 1) / ck; seg >= 0; --seg) {
    const int n0 = seg * ck, n1 = (n0 + ck < K) ? n0 + ck : K;
    AD_CK(cudaMemcpyAsync(segD, ckpt + (size_t)seg * m2, m2 * sizeof(double),
                          cudaMemcpyDeviceToDevice, s));
    for (int n = n0; n < n1; ++n) {
      const int j = n - n0;
      const double c = rec[(size_t)n * GCP_HISTORY_FIELDS + 5];
      const bool applied = c == c;  // NaN marks an identity step
      rs.stopped = 0;
      rs.apply = applied ? 1 : 0;
      if (applied) {
        const StepCoeffs k = step_coeffs(c, method);
        rs.a = k.a;
        rs.b = k.b;
        rs.g3 = k.g3;
      } else {
        rs.a = 1.0;
        rs.b = 0.0;
        rs.g3 = -2.0;
      }
      AD_CK(cudaMemcpyAsync(st, &rs, sizeof rs, cudaMemcpyHostToDevice, s));
      launch_f64_gemm1(segD + (size_t)j * m2, segS + (size_t)j * m2, M, M, nullptr, 1, M, part, st,
                       s);
      if (n + 1 < n1)
        launch_f64_gemm2(segS + (size_t)j * m2, segD + (size_t)j * m2, segD + (size_t)(j + 1) * m2,
                         M, M, st, s);
      // the replay state is read by the kernels just queued
      AD_CK(cudaStreamSynchronize(s));
    }
    for (int n = n1 - 1; n >= n0; --n) {
      const int j = n - n0;
      const double* Rc = rec.data() + (size_t)n * GCP_HISTORY_FIELDS;
      const double c = Rc[5];
      if (!(c == c)) continue;  // identity step: G passes through
      const double den = Rc[1] - Rc[2];
      const double* Dn = segD + (size_t)j * m2;
      const double* Sn = segS + (size_t)j * m2;
      const StepCoeffs k = step_coeffs(c, method);
      adj_gemm_kernel<<<nfull, kF64Threads, 0, s>>>(G, Dn, P, M, 0);  // P = G D
      adj_gemm_kernel<<<nfull, kF64Threads, 0, s>>>(G, Sn, Q, M, 0);  // Q = G D^2
      adj_gemm_kernel<<<nup, kF64Threads, 0, s>>>(Dn, P, R, M, 1);    // R = D G D
      // dL/dc = sum G o (a' D + b' S) + g3' sum Q o D
      adj_s_reduce_kernel<<<kRedBlocks, 256, 0, s>>>(G, Dn, Sn, k.dg3 != 0.0 ? Q : nullptr, k.da,
                                                     k.db, M, rpart);
      adj_reduce_finalize_kernel<<<1, 32, 0, s>>>(rpart, kRedBlocks, sc + 8);
      dim3 cg((M + 31) / 32, (M + 31) / 32);
      adj_combine_kernel<<<cg, dim3(32, 32), 0, s>>>(G, P, Q, R, Dn, Sn, Gn, M, k.a, k.b, k.g3,
                                                      k.dg3, c, den, sc + 8);
      AD_CK(cudaPeekAtLastError());
      double* t = G;
      G = Gn;
      Gn = t;
    }
  }
  // ---------------- guess ------------------------------------------------
  return adjoint_guess(H, M, N, ld, h_f64, guess, G, DK, gE, dLdH, gpart, st, s, err, errlen);
#undef AD_CK
  return GCP_OK;
}

}  // namespace gcp
