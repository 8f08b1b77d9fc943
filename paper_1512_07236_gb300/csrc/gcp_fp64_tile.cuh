// FP64 SIMT tile machinery shared by the FP64 products of the recursion and
// of its adjoint: a 256-thread CTA computes a BT x BT tile with an RT x RT
// register tile per thread, operands staged through shared memory in
// 16-deep K slices.
#pragma once
#include "gcp_internal.cuh"

namespace gcp {

constexpr int kF64Threads = 256;
constexpr int kF64BK = 16;

// Linear index over the tiles on or above the diagonal of a T x T tile grid.
__device__ __forceinline__ void f64_tile_coords(int t, int T, int& bi, int& bj) {
  int i = 0;
  while (t >= T - i) {
    t -= T - i;
    ++i;
  }
  bi = i;
  bj = i + t;
}

// acc[i][j] = sum_k A[m0 + ty + 16 i][k] * B[k][n0 + tx + 16 j].  A must be
// symmetric (its slice is read as rows A[k][m]); B is read by rows and may be
// any matrix.  Out-of-range elements read as zero.
template <int BT>
__device__ __forceinline__ void f64_mainloop(const double* __restrict__ A,
                                             const double* __restrict__ B, int M, int ld, int m0,
                                             int n0, double (&acc)[BT / 16][BT / 16],
                                             double (*As)[BT], double (*Bs)[BT]) {
  constexpr int RT = BT / 16;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < RT; ++i)
#pragma unroll
    for (int j = 0; j < RT; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < M; k0 += kF64BK) {
    for (int e = threadIdx.x; e < kF64BK * BT; e += kF64Threads) {
      const int k = e / BT, c = e % BT;
      const int gk = k0 + k;
      As[k][c] = (gk < M && m0 + c < M) ? A[(size_t)gk * ld + m0 + c] : 0.0;
      Bs[k][c] = (gk < M && n0 + c < M) ? B[(size_t)gk * ld + n0 + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kF64BK; ++k) {
      double a[RT], b[RT];
#pragma unroll
      for (int i = 0; i < RT; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < RT; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int j = 0; j < RT; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
}

}  // namespace gcp
