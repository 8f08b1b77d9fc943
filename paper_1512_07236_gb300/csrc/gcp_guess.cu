// Initial guess: the canonical guess (Eq. dmguess with the coefficients of
// Eq. pmcpguess), the mixed HPCP+ guess (Eq. hpcpguess, alpha from
// Eq. hpcpguessalpha) and the hole guess I - Dbar0.  All three are
//   D0 = theta I + b (mu I - H)
// with b = beta_min (canonical), b = beta_max (hole: I - Dbar0 with
// Dbar0 = thetabar I - beta_max (mu I - H)), or
// b = alpha beta_min + (1 - alpha) beta_max (HPCP+), where
// beta_min / beta_max are the smaller / larger of theta/(H_max - mu) and
// thetabar/(mu - H_min).
//
// Pass 1 (HBM-bound, one read of H): per row i the Gershgorin disc
//   [H_ii - r_i, H_ii + r_i], r_i = sum_{j != i} |H_ij|,
// reduced to H_min = min_i(H_ii - r_i), H_max = max_i(H_ii + r_i), Tr H,
// max|H_ii| and sum_{j != i} H_ij^2; one warp per row, per-block partials
// (deterministic order).
// Pass 2 (one block): mu = Tr H / M, theta = N/M, the betas and b.  For
// HPCP+, Tr D0^2 = M theta^2 + b^2 F with F = ||mu I - H||_F^2 (the trace of
// mu I - H vanishes), so the target of Eq. hpcpguessalpha fixes
// b^2 = (target - M theta^2) / F and alpha = (beta_max - b)/(beta_max -
// beta_min), clamped to [0, 1]; F is the off-diagonal sum of pass 1 plus
// sum_i (H_ii - mu)^2 read from the diagonal.
// Pass 3 (HBM-bound, read H once, write D0 once):
//   D0 = theta I + b (mu I - H), or the shifted X0 = D0 - theta J with
//   its split halves for the tensor-core path.
#include "gcp_device.cuh"
#include "gcp_internal.cuh"

namespace gcp {

namespace {
constexpr int kGuessThreads = 256;
constexpr int kGuessMaxBlocks = 1216;  // 8 x 152 SMs

// Per-row Gershgorin terms accumulated by one warp (lanes end identical).
template <typename T>
__device__ __forceinline__ void guess_row(const T* __restrict__ row, int i, int M, double& lo,
                                          double& hi, double& tr, double& mx, double& off2) {
  const int lane = threadIdx.x & 31;
  double r = 0.0, q = 0.0;
  for (int j = lane; j < M; j += 32) {
    const double h = (double)row[j];
    r += fabs(h);
    q += h * h;
  }
  r = warp_sum(r);
  q = warp_sum(q);
  const double d = (double)row[i];
  r -= fabs(d);
  lo = fmin(lo, d - r);
  hi = fmax(hi, d + r);
  tr += d;
  mx = fmax(mx, fabs(d));
  off2 += q - d * d;
}

// Combine the warps of a block in a fixed order into part[0..4].
__device__ __forceinline__ void guess_block_combine(double lo, double hi, double tr, double mx,
                                                    double off2, double* sh,
                                                    double* __restrict__ part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sh[warp * kGuessFields + 0] = lo;
    sh[warp * kGuessFields + 1] = hi;
    sh[warp * kGuessFields + 2] = tr;
    sh[warp * kGuessFields + 3] = mx;
    sh[warp * kGuessFields + 4] = off2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = INFINITY, b = -INFINITY, t = 0.0, m = 0.0, o = 0.0;
    for (int w = 0; w < kGuessThreads / 32; ++w) {
      a = fmin(a, sh[w * kGuessFields + 0]);
      b = fmax(b, sh[w * kGuessFields + 1]);
      t += sh[w * kGuessFields + 2];
      m = fmax(m, sh[w * kGuessFields + 3]);
      o += sh[w * kGuessFields + 4];
    }
    part[0] = a;
    part[1] = b;
    part[2] = t;
    part[3] = m;
    part[4] = o;
  }
}

template <typename T>
__global__ void __launch_bounds__(kGuessThreads) guess_reduce_kernel(const T* __restrict__ H,
                                                                      int M, int ld,
                                                                      double* __restrict__ part) {
  __shared__ double sh[32 * kGuessFields];
  const int warps_per_block = kGuessThreads / 32;
  const int gw = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
  const int nw = gridDim.x * warps_per_block;
  double lo = INFINITY, hi = -INFINITY, tr = 0.0, mx = 0.0, off2 = 0.0;
  for (int i = gw; i < M; i += nw) guess_row(H + (size_t)i * ld, i, M, lo, hi, tr, mx, off2);
  guess_block_combine(lo, hi, tr, mx, off2, sh, part + (size_t)blockIdx.x * kGuessFields);
}

// Guess coefficients into the state from the combined partials.
__device__ void guess_params(double lo, double hi, double tr, double mx, double F, int M, int N,
                             int mode, State* st) {
  const double theta = (double)N / (double)M;
  const double mu = tr / (double)M;
  // zero-width interval (H = mu I up to rounding): beta2 undefined
  const int no_gap = (hi - lo) <= 8.0 * (double)M * kU64 * fmax(1.0, mx);
  double b = 0.0, alpha = 1.0;
  if (!no_gap) {
    double bt = INFINITY, bb = INFINITY;
    if (hi - mu > 0.0) bt = theta / (hi - mu);
    if (mu - lo > 0.0) bb = (1.0 - theta) / (mu - lo);
    const double bmin = fmin(bt, bb), bmax = fmax(bt, bb);
    b = bmin;
    if (mode != GCP_GUESS_CANONICAL && isfinite(bmax)) {
      if (mode == GCP_GUESS_HOLE) {
        alpha = 0.0;
      } else {
        const double delta = 2.0 / 3.0, Md = (double)M, Nd = (double)N;
        double target = 0.0;
        bool has = true;
        if (theta <= 1.0 - delta)
          target = Nd - delta * Nd;
        else if (theta >= delta)
          target = Nd - delta * (Md - Nd);
        else
          has = false;
        alpha = 0.5;
        if (has && F > 0.0 && bmax > bmin) {
          const double b2 = (target - Md * theta * theta) / F;
          const double bt2 = b2 > 0.0 ? sqrt(b2) : 0.0;
          alpha = fmin(fmax((bmax - bt2) / (bmax - bmin), 0.0), 1.0);
        }
      }
      b = alpha * bmin + (1.0 - alpha) * bmax;
    }
  }
  st->mu = mu;
  st->beta2 = b;
  st->alpha = alpha;
  st->hmin = lo;
  st->hmax = hi;
  st->theta = theta;
  st->no_gap = no_gap;
}

template <typename T>
__global__ void __launch_bounds__(kGuessThreads) guess_finalize_kernel(
    const double* __restrict__ part, int nblocks, int M, int N, const T* __restrict__ H, int ld,
    int mode, State* st) {
  __shared__ double red[32];
  __shared__ double mu_sh;
  __shared__ double acc[kGuessFields];
  if (threadIdx.x == 0) {
    double lo = INFINITY, hi = -INFINITY, tr = 0.0, mx = 0.0, off2 = 0.0;
    for (int b = 0; b < nblocks; ++b) {
      const double* p = part + (size_t)b * kGuessFields;
      lo = fmin(lo, p[0]);
      hi = fmax(hi, p[1]);
      tr += p[2];
      mx = fmax(mx, p[3]);
      off2 += p[4];
    }
    acc[0] = lo;
    acc[1] = hi;
    acc[2] = tr;
    acc[3] = mx;
    acc[4] = off2;
    mu_sh = tr / (double)M;
  }
  __syncthreads();
  double v[1] = {0.0};
  if (mode == GCP_GUESS_HPCP_PLUS) {
    const double mu = mu_sh;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
      const double d = (double)H[(size_t)i * ld + i] - mu;
      v[0] += d * d;
    }
  }
  block_sum<1>(v, red);
  if (threadIdx.x == 0) guess_params(acc[0], acc[1], acc[2], acc[3], acc[4] + v[0], M, N, mode, st);
}

template <typename T, typename O>
__global__ void guess_write_d_kernel(const T* __restrict__ H, int M, int ld, O* __restrict__ D,
                                     int ldd, int rows_pad, const State* __restrict__ st) {
  const double beta2 = st->beta2, mu = st->mu, theta = st->theta;
  const int i = blockIdx.y;
  if (i >= rows_pad) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < rows_pad; j += gridDim.x * blockDim.x) {
    double v = 0.0;
    if (i < M && j < M) {
      v = -beta2 * (double)H[(size_t)i * ld + j];
      if (i == j) v += theta + beta2 * mu;
    }
    D[(size_t)i * ldd + j] = (O)v;
  }
}

template <typename T, bool BF16>
__global__ void guess_write_x_kernel(const T* __restrict__ H, int M, int ld, float* __restrict__ X,
                                     typename Split<BF16>::T* __restrict__ Xh,
                                     typename Split<BF16>::T* __restrict__ Xl, int Mp,
                                     float scale, const State* __restrict__ st) {
  const double beta2 = st->beta2, mu = st->mu;
  const int i = blockIdx.y;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < Mp; j += gridDim.x * blockDim.x) {
    double v = 0.0;
    if (i < M && j < M) {
      // the upper triangle of H only: the split state is exactly symmetric
      // (the tensor-core epilogues write each mirrored element from the
      // same inputs as the direct one)
      v = -beta2 * (double)(i <= j ? H[(size_t)i * ld + j] : H[(size_t)j * ld + i]);
      if (i == j) v += beta2 * mu;
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
}  // namespace

// max_{i<j} |H_ij - H_ji| and max_ij |H_ij|: one row i per block.y, the
// columns j > i of that row against column i below the diagonal; block
// maxima go to out[] with an integer atomicMax on the bit patterns (for
// non-negative doubles the order of the bits is the order of the values).
template <typename T>
__global__ void sym_check_kernel(const T* __restrict__ H, int M, int ld,
                                 unsigned long long* __restrict__ out) {
  const int i = blockIdx.y;
  double asym = 0.0, amax = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
    const double a = (double)H[(size_t)i * ld + j];
    amax = fmax(amax, fabs(a));
    if (j > i) asym = fmax(asym, fabs(a - (double)H[(size_t)j * ld + i]));
  }
  asym = warp_max(asym);
  amax = warp_max(amax);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], (unsigned long long)__double_as_longlong(asym));
    atomicMax(&out[1], (unsigned long long)__double_as_longlong(amax));
  }
}

int guess_partial_blocks(int M) {
  int b = (M + (kGuessThreads / 32) - 1) / (kGuessThreads / 32);
  return b < kGuessMaxBlocks ? b : kGuessMaxBlocks;
}

void launch_sym_check(const void* H, int h_f64, int M, int ld, double* out, cudaStream_t s) {
  cudaMemsetAsync(out, 0, 2 * sizeof(double), s);
  dim3 grid((M + 255) / 256 < 8 ? (M + 255) / 256 : 8, M);
  if (h_f64)
    sym_check_kernel<double><<<grid, 256, 0, s>>>((const double*)H, M, ld,
                                                  (unsigned long long*)out);
  else
    sym_check_kernel<float><<<grid, 256, 0, s>>>((const float*)H, M, ld, (unsigned long long*)out);
}

void launch_guess_reduce(const void* H, int h_f64, int M, int ld, double* part, cudaStream_t s) {
  const int nb = guess_partial_blocks(M);
  if (h_f64)
    guess_reduce_kernel<double><<<nb, kGuessThreads, 0, s>>>((const double*)H, M, ld, part);
  else
    guess_reduce_kernel<float><<<nb, kGuessThreads, 0, s>>>((const float*)H, M, ld, part);
}

void launch_guess_finalize(const double* part, int nblocks, int M, int N, const void* H,
                           int h_f64, int ld, int guess_mode, State* st, cudaStream_t s) {
  if (h_f64)
    guess_finalize_kernel<double><<<1, kGuessThreads, 0, s>>>(part, nblocks, M, N,
                                                             (const double*)H, ld, guess_mode, st);
  else
    guess_finalize_kernel<float><<<1, kGuessThreads, 0, s>>>(part, nblocks, M, N,
                                                            (const float*)H, ld, guess_mode, st);
}

void launch_guess_write_d(const void* H, int h_f64, int M, int ld, void* D, int d_f64, int ldd,
                          int rows_pad, const State* st, cudaStream_t s) {
  dim3 grid((rows_pad + 255) / 256 < 8 ? (rows_pad + 255) / 256 : 8, rows_pad);
  if (h_f64 && d_f64)
    guess_write_d_kernel<double, double><<<grid, 256, 0, s>>>((const double*)H, M, ld, (double*)D,
                                                             ldd, rows_pad, st);
  else if (h_f64)
    guess_write_d_kernel<double, float><<<grid, 256, 0, s>>>((const double*)H, M, ld, (float*)D,
                                                            ldd, rows_pad, st);
  else if (d_f64)
    guess_write_d_kernel<float, double><<<grid, 256, 0, s>>>((const float*)H, M, ld, (double*)D,
                                                            ldd, rows_pad, st);
  else
    guess_write_d_kernel<float, float><<<grid, 256, 0, s>>>((const float*)H, M, ld, (float*)D, ldd,
                                                           rows_pad, st);
}

void launch_guess_write_x(const void* H, int h_f64, int M, int ld, float* X, void* Xh, void* Xl,
                          int Mp, int bf16, float split_scale, const State* st, cudaStream_t s) {
  dim3 grid((Mp + 255) / 256 < 8 ? (Mp + 255) / 256 : 8, Mp);
  if (bf16) {
    using T = Split<true>::T;
    if (h_f64)
      guess_write_x_kernel<double, true><<<grid, 256, 0, s>>>((const double*)H, M, ld, X, (T*)Xh,
                                                             (T*)Xl, Mp, split_scale, st);
    else
      guess_write_x_kernel<float, true><<<grid, 256, 0, s>>>((const float*)H, M, ld, X, (T*)Xh,
                                                            (T*)Xl, Mp, split_scale, st);
  } else {
    using T = Split<false>::T;
    if (h_f64)
      guess_write_x_kernel<double, false><<<grid, 256, 0, s>>>((const double*)H, M, ld, X, (T*)Xh,
                                                              (T*)Xl, Mp, split_scale, st);
    else
      guess_write_x_kernel<float, false><<<grid, 256, 0, s>>>((const float*)H, M, ld, X, (T*)Xh,
                                                             (T*)Xl, Mp, split_scale, st);
  }
}

}  // namespace gcp

// ---- batched guess: one launch per pass over all instances ---------------
namespace gcp {
namespace {
template <typename T>
__global__ void __launch_bounds__(kGuessThreads) batch_guess_reduce_kernel(
    const BatchItem* items, double* __restrict__ gpart) {
  __shared__ double sh[32 * kGuessFields];
  const BatchItem& it = items[blockIdx.y];
  if ((int)blockIdx.x >= it.gblocks) return;  // this instance uses gblocks blocks
  const T* H = (const T*)it.H;
  const int M = it.M, ld = it.ld;
  const int warps_per_block = kGuessThreads / 32;
  const int gw = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
  const int nw = it.gblocks * warps_per_block;
  double lo = INFINITY, hi = -INFINITY, tr = 0.0, mx = 0.0, off2 = 0.0;
  for (int i = gw; i < M; i += nw) guess_row(H + (size_t)i * ld, i, M, lo, hi, tr, mx, off2);
  guess_block_combine(lo, hi, tr, mx, off2, sh,
                      gpart + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * kGuessFields);
}

// One block per instance: the same combination as a single solve's
// guess_finalize_kernel (partials in block order, the HPCP+ diagonal sum
// as a block reduction), so both give the same coefficients.
template <typename T>
__global__ void __launch_bounds__(kGuessThreads) batch_guess_finalize_kernel(
    const BatchItem* items, const double* __restrict__ gpart, int gstride, int mode) {
  const BatchItem& it = items[blockIdx.x];
  __shared__ double red[32];
  __shared__ double mu_sh;
  __shared__ double acc[kGuessFields];
  if (threadIdx.x == 0) {
    double lo = INFINITY, hi = -INFINITY, tr = 0.0, mx = 0.0, off2 = 0.0;
    for (int k = 0; k < it.gblocks; ++k) {
      const double* p = gpart + ((size_t)blockIdx.x * gstride + k) * kGuessFields;
      lo = fmin(lo, p[0]);
      hi = fmax(hi, p[1]);
      tr += p[2];
      mx = fmax(mx, p[3]);
      off2 += p[4];
    }
    acc[0] = lo;
    acc[1] = hi;
    acc[2] = tr;
    acc[3] = mx;
    acc[4] = off2;
    mu_sh = tr / (double)it.M;
  }
  __syncthreads();
  double v[1] = {0.0};
  if (mode == GCP_GUESS_HPCP_PLUS) {
    const T* H = (const T*)it.H;
    const double mu = mu_sh;
    for (int i = threadIdx.x; i < it.M; i += blockDim.x) {
      const double d = (double)H[(size_t)i * it.ld + i] - mu;
      v[0] += d * d;
    }
  }
  block_sum<1>(v, red);
  if (threadIdx.x == 0)
    guess_params(acc[0], acc[1], acc[2], acc[3], acc[4] + v[0], it.M, it.N, mode, it.st);
}

template <typename T, bool BF16>
__global__ void batch_guess_write_x_kernel(const BatchItem* items, float scale) {
  const BatchItem& it = items[blockIdx.y];
  const T* H = (const T*)it.H;
  const double beta2 = it.st->beta2, mu = it.st->mu;
  using HT = typename Split<BF16>::T;
  const size_t n = (size_t)it.Mp * it.Mp;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / it.Mp), j = (int)(e % it.Mp);
    double v = 0.0;
    if (i < it.M && j < it.M) {
      // the upper triangle of H only (exactly symmetric split state)
      v = -beta2 * (double)(i <= j ? H[(size_t)i * it.ld + j] : H[(size_t)j * it.ld + i]);
      if (i == j) v += beta2 * mu;
    }
    const float x = (float)v;
    const size_t o = (size_t)i * it.Mp + j;
    it.X[0][o] = x;
    HT h, l;
    Split<BF16>::split(x * scale, h, l);
    ((HT*)it.Xh[0])[o] = h;
    ((HT*)it.Xl[0])[o] = l;
  }
}

template <typename T>
__global__ void batch_guess_write_d_kernel(const BatchItem* items) {
  const BatchItem& it = items[blockIdx.y];
  const T* H = (const T*)it.H;
  const double beta2 = it.st->beta2, mu = it.st->mu, theta = it.st->theta;
  const size_t n = (size_t)it.M * it.M;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / it.M), j = (int)(e % it.M);
    double v = -beta2 * (double)H[(size_t)i * it.ld + j];
    if (i == j) v += theta + beta2 * mu;
    it.D64[0][e] = v;
  }
}
}  // namespace

void launch_batch_guess(const BatchItem* items, int batch, int maxM, int h_f64, int split,
                        int bf16, float split_scale, double* gpart, int gstride, int guess_mode,
                        cudaStream_t s) {
  dim3 gr(gstride, batch);
  if (h_f64)
    batch_guess_reduce_kernel<double><<<gr, kGuessThreads, 0, s>>>(items, gpart);
  else
    batch_guess_reduce_kernel<float><<<gr, kGuessThreads, 0, s>>>(items, gpart);
  if (h_f64)
    batch_guess_finalize_kernel<double><<<batch, kGuessThreads, 0, s>>>(items, gpart, gstride,
                                                                        guess_mode);
  else
    batch_guess_finalize_kernel<float><<<batch, kGuessThreads, 0, s>>>(items, gpart, gstride,
                                                                       guess_mode);
  // blocks per instance: ~32 elements a thread for the largest instance
  auto ew = [](long long n) {
    const long long b = (n + 8191) / 8192;
    return (int)(b < 1 ? 1 : (b > 64 ? 64 : b));
  };
  if (split) {
    const int maxMp = tc_pad(maxM);
    dim3 g(ew((long long)maxMp * maxMp), batch);
    if (bf16) {
      if (h_f64)
        batch_guess_write_x_kernel<double, true><<<g, 256, 0, s>>>(items, split_scale);
      else
        batch_guess_write_x_kernel<float, true><<<g, 256, 0, s>>>(items, split_scale);
    } else {
      if (h_f64)
        batch_guess_write_x_kernel<double, false><<<g, 256, 0, s>>>(items, split_scale);
      else
        batch_guess_write_x_kernel<float, false><<<g, 256, 0, s>>>(items, split_scale);
    }
  } else {
    dim3 g(ew((long long)maxM * maxM), batch);
    if (h_f64)
      batch_guess_write_d_kernel<double><<<g, 256, 0, s>>>(items);
    else
      batch_guess_write_d_kernel<float><<<g, 256, 0, s>>>(items);
  }
}
}  // namespace gcp
