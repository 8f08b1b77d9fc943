// FP64 products of one GCP step with fused epilogues (the plain FP64 GPU
// path and the refinement engine of the mixed modes).
//
// GB300 runs FP64 on SIMT DFMA units at a small fraction of its tensor
// rate, so these kernels are DFMA-bound at any practical size: register
// tiles of RT x RT outputs per thread, operand slices staged in shared
// memory.  Only tiles on or above the diagonal are computed (the products
// of symmetric commuting matrices are symmetric); every element above the
// diagonal is stored twice (direct and mirrored), so the results are exactly
// symmetric.
//
// GEMM1 (S = D D) epilogue, per tile, in FP64 (Eq. mcwgamb, Eq. mcw1b):
//   T1 += D_ii, T2 += S_ii                 (diagonal tiles)
//   T3 += w S_ij D_ij                      (Tr D^3 for symmetric D)
//   R2 += w (S_ij - D_ij)^2                (||D^2 - D||_F^2, elementwise)
//   E  += w D_ij H_ij                      (Tr H D)
// over the upper triangle, with w = 2 above the diagonal (the element
// stands for its mirror) and 1 on it.  One record of partials per tile; the control kernel sums
// them in tile order, so the result does not depend on scheduling.
// GEMM2 (P = S D) epilogue: D_{n+1} = a D + b S + g3 P with the step's
// coefficients from the state (HPCP, Eq. hpcp3 expanded: a = 1 - 2c,
// b = 2 + 2c, g3 = -2; PMCP: Eq. pm1).
#include "gcp_device.cuh"
#include "gcp_fp64_tile.cuh"
#include "gcp_internal.cuh"

namespace gcp {

namespace {
constexpr int kThreads = kF64Threads;
constexpr int kBK = kF64BK;

__device__ __forceinline__ void tile_coords(int t, int T, int& bi, int& bj) {
  f64_tile_coords(t, T, bi, bj);
}

template <int BT, typename HT>
__global__ void __launch_bounds__(kThreads) f64_gemm1_kernel(const double* __restrict__ D,
                                                             double* __restrict__ S, int M, int ld,
                                                             const HT* __restrict__ H, int ldh,
                                                             double* __restrict__ part,
                                                             const State* __restrict__ st) {
  if (st->stopped) return;
  __shared__ double As[kBK][BT];
  __shared__ double Bs[kBK][BT];
  __shared__ double red[32 * 5];
  constexpr int RT = BT / 16;
  const int T = (M + BT - 1) / BT;
  int bi, bj;
  tile_coords(blockIdx.x, T, bi, bj);
  const int m0 = bi * BT, n0 = bj * BT;
  double acc[RT][RT];
  f64_mainloop<BT>(D, D, M, ld, m0, n0, acc, As, Bs);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int i = 0; i < RT; ++i) {
    const int r = m0 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < RT; ++j) {
      const int c = n0 + tx + 16 * j;
      // upper triangle only (weight 2 stands for the mirror), so the
      // stored result is exactly symmetric
      if (r < M && c < M && c >= r) {
        const double w = (c == r) ? 1.0 : 2.0;
        const double s = acc[i][j];
        const double d = D[(size_t)r * ld + c];
        if (r == c) {
          v[0] += d;
          v[1] += s;
        }
        v[2] += w * s * d;
        v[3] += w * (s - d) * (s - d);
        if (H) v[4] += w * d * (double)H[(size_t)r * ldh + c];
        S[(size_t)r * ld + c] = s;
        if (c != r) S[(size_t)c * ld + r] = s;
      }
    }
  }
  block_sum<5>(v, red);
  if (threadIdx.x == 0) {
    double* p = part + (size_t)blockIdx.x * kPartFields;
    p[0] = v[0];
    p[1] = v[1];
    p[2] = v[2];
    p[3] = v[3];
    p[4] = v[4];
    p[5] = 0.0;
  }
}

template <int BT>
__global__ void __launch_bounds__(kThreads) f64_gemm2_kernel(const double* __restrict__ S,
                                                             const double* __restrict__ D,
                                                             double* __restrict__ Dn, int M,
                                                             int ld, const State* __restrict__ st) {
  if (st->stopped) return;
  __shared__ double As[kBK][BT];
  __shared__ double Bs[kBK][BT];
  constexpr int RT = BT / 16;
  const int T = (M + BT - 1) / BT;
  int bi, bj;
  tile_coords(blockIdx.x, T, bi, bj);
  const int m0 = bi * BT, n0 = bj * BT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const bool apply = st->apply != 0;
  const double a = st->a, b = st->b, g3 = st->g3;
  double acc[RT][RT];
  if (apply) {
    f64_mainloop<BT>(S, D, M, ld, m0, n0, acc, As, Bs);
  }
#pragma unroll
  for (int i = 0; i < RT; ++i) {
    const int r = m0 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < RT; ++j) {
      const int c = n0 + tx + 16 * j;
      if (r < M && c < M && c >= r) {
        const size_t o = (size_t)r * ld + c;
        const double d = D[o];
        const double x = apply ? (a * d + b * S[o] + g3 * acc[i][j]) : d;
        Dn[o] = x;
        if (c != r) Dn[(size_t)c * ld + r] = x;
      }
    }
  }
}
}  // namespace

int f64_tile(int M) { return M <= 1024 ? 32 : 64; }

int f64_num_tiles(int M) {
  const int BT = f64_tile(M);
  const int T = (M + BT - 1) / BT;
  return T * (T + 1) / 2;
}

void launch_f64_gemm1(const double* D, double* S, int M, int ld, const void* H, int h_f64, int ldh,
                      double* part, const State* st, cudaStream_t s) {
  const int nt = f64_num_tiles(M);
  if (f64_tile(M) == 32) {
    if (h_f64 || !H)
      f64_gemm1_kernel<32, double><<<nt, kThreads, 0, s>>>(D, S, M, ld, (const double*)H, ldh, part,
                                                          st);
    else
      f64_gemm1_kernel<32, float><<<nt, kThreads, 0, s>>>(D, S, M, ld, (const float*)H, ldh, part,
                                                         st);
  } else {
    if (h_f64 || !H)
      f64_gemm1_kernel<64, double><<<nt, kThreads, 0, s>>>(D, S, M, ld, (const double*)H, ldh, part,
                                                          st);
    else
      f64_gemm1_kernel<64, float><<<nt, kThreads, 0, s>>>(D, S, M, ld, (const float*)H, ldh, part,
                                                         st);
  }
}

void launch_f64_gemm2(const double* S, const double* D, double* Dn, int M, int ld,
                      const State* st, cudaStream_t s) {
  const int nt = f64_num_tiles(M);
  if (f64_tile(M) == 32)
    f64_gemm2_kernel<32><<<nt, kThreads, 0, s>>>(S, D, Dn, M, ld, st);
  else
    f64_gemm2_kernel<64><<<nt, kThreads, 0, s>>>(S, D, Dn, M, ld, st);
}

// ---- batched: one launch over the tiles of every instance ----------------
// tile_inst[t] names the instance of work-list tile t; the instance's tiles
// are the 32 x 32 upper tiles of its matrix, in the order of tile_coords.
namespace {
constexpr int kBT = 32;

__global__ void __launch_bounds__(kThreads) batch_f64_gemm1_kernel(const BatchItem* items,
                                                                   const int* tile_inst,
                                                                   double* __restrict__ part) {
  const BatchItem& it = items[tile_inst[blockIdx.x]];
  State* st = it.st;
  if (st->stopped) return;
  __shared__ double As[kBK][kBT];
  __shared__ double Bs[kBK][kBT];
  __shared__ double red[32 * 5];
  constexpr int RT = kBT / 16;
  const int M = it.M, ld = it.M;
  const double* D = it.D64[st->parity];
  double* S = it.S64;
  const int T = (M + kBT - 1) / kBT;
  int bi, bj;
  tile_coords(blockIdx.x - it.f64_off, T, bi, bj);
  const int m0 = bi * kBT, n0 = bj * kBT;
  double acc[RT][RT];
  f64_mainloop<kBT>(D, D, M, ld, m0, n0, acc, As, Bs);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int i = 0; i < RT; ++i) {
    const int r = m0 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < RT; ++j) {
      const int c = n0 + tx + 16 * j;
      if (r < M && c < M && c >= r) {
        const double w = (c == r) ? 1.0 : 2.0;
        const double s = acc[i][j];
        const double d = D[(size_t)r * ld + c];
        if (r == c) {
          v[0] += d;
          v[1] += s;
        }
        v[2] += w * s * d;
        v[3] += w * (s - d) * (s - d);
        S[(size_t)r * ld + c] = s;
        if (c != r) S[(size_t)c * ld + r] = s;
      }
    }
  }
  block_sum<5>(v, red);
  if (threadIdx.x == 0) {
    double* p = part + (size_t)blockIdx.x * kPartFields;
    p[0] = v[0];
    p[1] = v[1];
    p[2] = v[2];
    p[3] = v[3];
    p[4] = 0.0;
    p[5] = 0.0;
  }
}

__global__ void __launch_bounds__(kThreads) batch_f64_gemm2_kernel(const BatchItem* items,
                                                                   const int* tile_inst) {
  const BatchItem& it = items[tile_inst[blockIdx.x]];
  const State* st = it.st;
  if (st->stopped) return;
  __shared__ double As[kBK][kBT];
  __shared__ double Bs[kBK][kBT];
  constexpr int RT = kBT / 16;
  const int M = it.M, ld = it.M;
  // the control kernel has flipped the parity for this step
  const double* D = it.D64[st->parity ^ 1];
  double* Dn = it.D64[st->parity];
  const double* S = it.S64;
  const int T = (M + kBT - 1) / kBT;
  int bi, bj;
  tile_coords(blockIdx.x - it.f64_off, T, bi, bj);
  const int m0 = bi * kBT, n0 = bj * kBT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const bool apply = st->apply != 0;
  const double a = st->a, b = st->b, g3 = st->g3;
  double acc[RT][RT];
  if (apply) f64_mainloop<kBT>(S, D, M, ld, m0, n0, acc, As, Bs);
#pragma unroll
  for (int i = 0; i < RT; ++i) {
    const int r = m0 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < RT; ++j) {
      const int c = n0 + tx + 16 * j;
      if (r < M && c < M && c >= r) {
        const size_t o = (size_t)r * ld + c;
        const double d = D[o];
        const double x = apply ? (a * d + b * S[o] + g3 * acc[i][j]) : d;
        Dn[o] = x;
        if (c != r) Dn[(size_t)c * ld + r] = x;
      }
    }
  }
}
}  // namespace

int batch_f64_tiles(int M) {
  const int T = (M + kBT - 1) / kBT;
  return T * (T + 1) / 2;
}

void launch_batch_f64_gemm1(const BatchItem* items, int batch, const int* tile_inst, int ntiles,
                            double* part, cudaStream_t s) {
  (void)batch;
  batch_f64_gemm1_kernel<<<ntiles, kThreads, 0, s>>>(items, tile_inst, part);
}

void launch_batch_f64_gemm2(const BatchItem* items, int batch, const int* tile_inst, int ntiles,
                            cudaStream_t s) {
  (void)batch;
  batch_f64_gemm2_kernel<<<ntiles, kThreads, 0, s>>>(items, tile_inst);
}

}  // namespace gcp
