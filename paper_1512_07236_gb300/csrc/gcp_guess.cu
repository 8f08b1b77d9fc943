// Canonical initial guess (Eq. dmguess with the coefficients of Eq. pmcpguess).
//
// Pass 1 (HBM-bound, one read of H): per row i the Gershgorin disc
//   [H_ii - r_i, H_ii + r_i], r_i = sum_{j != i} |H_ij|,
// reduced to H_min = min_i(H_ii - r_i), H_max = max_i(H_ii + r_i), Tr H and
// max|H_ii|; one warp per row, per-block partials (deterministic order).
// Pass 2 (one block): mu = Tr H / M, theta = N/M,
//   beta2 = min{theta/(H_max - mu), (1-theta)/(mu - H_min)}.
// Pass 3 (HBM-bound, read H once, write D0 once):
//   D0 = theta I + beta2 (mu I - H), or the shifted X0 = D0 - theta J with
//   its split halves for the tensor-core path.
#include "gcp_device.cuh"
#include "gcp_internal.cuh"

namespace gcp {

namespace {
constexpr int kGuessThreads = 256;
constexpr int kGuessMaxBlocks = 1216;  // 8 x 152 SMs

template <typename T>
__global__ void __launch_bounds__(kGuessThreads) guess_reduce_kernel(const T* __restrict__ H,
                                                                      int M, int ld,
                                                                      double* __restrict__ part) {
  __shared__ double sh[32 * 4];
  const int lane = threadIdx.x & 31;
  const int warps_per_block = kGuessThreads / 32;
  const int gw = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
  const int nw = gridDim.x * warps_per_block;
  double lo = INFINITY, hi = -INFINITY, tr = 0.0, mx = 0.0;
  for (int i = gw; i < M; i += nw) {
    const T* row = H + (size_t)i * ld;
    double r = 0.0;
    for (int j = lane; j < M; j += 32) r += fabs((double)row[j]);
    r = warp_sum(r);
    const double d = (double)row[i];
    r -= fabs(d);
    lo = fmin(lo, d - r);
    hi = fmax(hi, d + r);
    tr += d;  // identical in every lane
    mx = fmax(mx, fabs(d));
  }
  // lanes hold identical values; combine warps in a fixed order
  const int warp = threadIdx.x >> 5;
  if (lane == 0) {
    sh[warp * 4 + 0] = lo;
    sh[warp * 4 + 1] = hi;
    sh[warp * 4 + 2] = tr;
    sh[warp * 4 + 3] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = INFINITY, b = -INFINITY, t = 0.0, m = 0.0;
    for (int w = 0; w < warps_per_block; ++w) {
      a = fmin(a, sh[w * 4 + 0]);
      b = fmax(b, sh[w * 4 + 1]);
      t += sh[w * 4 + 2];
      m = fmax(m, sh[w * 4 + 3]);
    }
    part[blockIdx.x * 4 + 0] = a;
    part[blockIdx.x * 4 + 1] = b;
    part[blockIdx.x * 4 + 2] = t;
    part[blockIdx.x * 4 + 3] = m;
  }
}

__global__ void guess_finalize_kernel(const double* __restrict__ part, int nblocks, int M, int N,
                                      State* st) {
  if (threadIdx.x != 0) return;
  double lo = INFINITY, hi = -INFINITY, tr = 0.0, mx = 0.0;
  for (int b = 0; b < nblocks; ++b) {
    lo = fmin(lo, part[b * 4 + 0]);
    hi = fmax(hi, part[b * 4 + 1]);
    tr += part[b * 4 + 2];
    mx = fmax(mx, part[b * 4 + 3]);
  }
  const double theta = (double)N / (double)M;
  const double mu = tr / (double)M;
  // zero-width interval (H = mu I up to rounding): beta2 undefined
  const int no_gap = (hi - lo) <= 8.0 * (double)M * kU64 * fmax(1.0, mx);
  double beta2 = 0.0;
  if (!no_gap) {
    double bt = INFINITY, bb = INFINITY;
    if (hi - mu > 0.0) bt = theta / (hi - mu);
    if (mu - lo > 0.0) bb = (1.0 - theta) / (mu - lo);
    beta2 = fmin(bt, bb);
  }
  st->mu = mu;
  st->beta2 = beta2;
  st->hmin = lo;
  st->hmax = hi;
  st->theta = theta;
  st->no_gap = no_gap;
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
      v = -beta2 * (double)H[(size_t)i * ld + j];
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

int guess_partial_blocks(int M) {
  int b = (M + (kGuessThreads / 32) - 1) / (kGuessThreads / 32);
  return b < kGuessMaxBlocks ? b : kGuessMaxBlocks;
}

void launch_guess_reduce(const void* H, int h_f64, int M, int ld, double* part, cudaStream_t s) {
  const int nb = guess_partial_blocks(M);
  if (h_f64)
    guess_reduce_kernel<double><<<nb, kGuessThreads, 0, s>>>((const double*)H, M, ld, part);
  else
    guess_reduce_kernel<float><<<nb, kGuessThreads, 0, s>>>((const float*)H, M, ld, part);
}

void launch_guess_finalize(const double* part, int nblocks, int M, int N, State* st,
                           cudaStream_t s) {
  guess_finalize_kernel<<<1, 32, 0, s>>>(part, nblocks, M, N, st);
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
  __shared__ double sh[32 * 4];
  const BatchItem& it = items[blockIdx.y];
  if ((int)blockIdx.x >= it.gblocks) return;  // this instance uses gblocks blocks
  const T* H = (const T*)it.H;
  const int M = it.M, ld = it.ld;
  const int lane = threadIdx.x & 31;
  const int warps_per_block = kGuessThreads / 32;
  const int gw = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
  const int nw = it.gblocks * warps_per_block;
  double lo = INFINITY, hi = -INFINITY, tr = 0.0, mx = 0.0;
  for (int i = gw; i < M; i += nw) {
    const T* row = H + (size_t)i * ld;
    double r = 0.0;
    for (int j = lane; j < M; j += 32) r += fabs((double)row[j]);
    r = warp_sum(r);
    const double d = (double)row[i];
    r -= fabs(d);
    lo = fmin(lo, d - r);
    hi = fmax(hi, d + r);
    tr += d;
    mx = fmax(mx, fabs(d));
  }
  const int warp = threadIdx.x >> 5;
  if (lane == 0) {
    sh[warp * 4 + 0] = lo;
    sh[warp * 4 + 1] = hi;
    sh[warp * 4 + 2] = tr;
    sh[warp * 4 + 3] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = INFINITY, b = -INFINITY, t = 0.0, m = 0.0;
    for (int w = 0; w < warps_per_block; ++w) {
      a = fmin(a, sh[w * 4 + 0]);
      b = fmax(b, sh[w * 4 + 1]);
      t += sh[w * 4 + 2];
      m = fmax(m, sh[w * 4 + 3]);
    }
    double* p = gpart + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 4;
    p[0] = a;
    p[1] = b;
    p[2] = t;
    p[3] = m;
  }
}

__global__ void batch_guess_finalize_kernel(const BatchItem* items, int batch,
                                            const double* __restrict__ gpart, int gstride) {
  const int bi = blockIdx.x * blockDim.x + threadIdx.x;
  if (bi >= batch) return;
  const BatchItem& it = items[bi];
  State* st = it.st;
  double lo = INFINITY, hi = -INFINITY, tr = 0.0, mx = 0.0;
  for (int k = 0; k < it.gblocks; ++k) {
    const double* p = gpart + ((size_t)bi * gstride + k) * 4;
    lo = fmin(lo, p[0]);
    hi = fmax(hi, p[1]);
    tr += p[2];
    mx = fmax(mx, p[3]);
  }
  const int M = it.M, N = it.N;
  const double theta = (double)N / (double)M;
  const double mu = tr / (double)M;
  const int no_gap = (hi - lo) <= 8.0 * (double)M * kU64 * fmax(1.0, mx);
  double beta2 = 0.0;
  if (!no_gap) {
    double bt = INFINITY, bb = INFINITY;
    if (hi - mu > 0.0) bt = theta / (hi - mu);
    if (mu - lo > 0.0) bb = (1.0 - theta) / (mu - lo);
    beta2 = fmin(bt, bb);
  }
  st->mu = mu;
  st->beta2 = beta2;
  st->hmin = lo;
  st->hmax = hi;
  st->theta = theta;
  st->no_gap = no_gap;
}

template <typename T, bool BF16>
__global__ void batch_guess_write_x_kernel(const BatchItem* items, float scale) {
  const BatchItem& it = items[blockIdx.z];
  const int i = blockIdx.y;
  if (i >= it.Mp) return;
  const T* H = (const T*)it.H;
  const double beta2 = it.st->beta2, mu = it.st->mu;
  using HT = typename Split<BF16>::T;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < it.Mp; j += gridDim.x * blockDim.x) {
    double v = 0.0;
    if (i < it.M && j < it.M) {
      v = -beta2 * (double)H[(size_t)i * it.ld + j];
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
  const BatchItem& it = items[blockIdx.z];
  const int i = blockIdx.y;
  if (i >= it.M) return;
  const T* H = (const T*)it.H;
  const double beta2 = it.st->beta2, mu = it.st->mu, theta = it.st->theta;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < it.M; j += gridDim.x * blockDim.x) {
    double v = -beta2 * (double)H[(size_t)i * it.ld + j];
    if (i == j) v += theta + beta2 * mu;
    it.D64[0][(size_t)i * it.M + j] = v;
  }
}
}  // namespace

void launch_batch_guess(const BatchItem* items, int batch, int maxM, int h_f64, int split,
                        int bf16, float split_scale, double* gpart, int gstride, cudaStream_t s) {
  dim3 gr(gstride, batch);
  if (h_f64)
    batch_guess_reduce_kernel<double><<<gr, kGuessThreads, 0, s>>>(items, gpart);
  else
    batch_guess_reduce_kernel<float><<<gr, kGuessThreads, 0, s>>>(items, gpart);
  batch_guess_finalize_kernel<<<(batch + 127) / 128, 128, 0, s>>>(items, batch, gpart, gstride);
  if (split) {
    const int maxMp = ((maxM + 255) / 256) * 256;
    dim3 g((maxMp + 255) / 256 < 4 ? (maxMp + 255) / 256 : 4, maxMp, batch);
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
    dim3 g((maxM + 255) / 256 < 4 ? (maxM + 255) / 256 : 4, maxM, batch);
    if (h_f64)
      batch_guess_write_d_kernel<double><<<g, 256, 0, s>>>(items);
    else
      batch_guess_write_d_kernel<float><<<g, 256, 0, s>>>(items);
  }
}
}  // namespace gcp
