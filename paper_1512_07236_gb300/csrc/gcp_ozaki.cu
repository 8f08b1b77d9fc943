// Exact slice products for the FP64 refinement of the mixed modes.
//
// GB300 runs FP64 on SIMT units at ~1.2 TFLOP/s; one FP64 D^2 at M = 8192
// takes ~0.45 s.  Here D^2 is formed on the tensor cores without rounding:
//   * each row i of D is scaled by 2^e_i with |D_ij| <= 2^e_i / 2 and cut
//     into ns signed digits of b bits, D_ij = 2^e_i sum_s d_s B^-(s+1) + r,
//     B = 2^b, |d_s| <= B/2, |r| <= 2^e_i B^-ns / 2; digits are small
//     integers, exact in fp16.  M <= 16384: b = 6, ns = 8 (48-bit fixed
//     point); larger M: b = 5, ns = 9 (45 bits);
//   * (D D)_ij = 2^(e_i+e_j) sum_w B^-(w+2) sum_{s+t=w} sum_k d_s(i,k) d_t(j,k)
//     over the weights w kept: at most w = 0..ns (b = 6: 43 pairs; b = 5:
//     53), fewer when the refinement's tolerance allows (oz_weight_cap).
//     The dropped weights have random signs except on the diagonal, where
//     the dropped squares d_s(i,k)^2 are always positive; the diagonal is
//     therefore not taken from this product but formed in FP64 by the
//     finalize pass (finalize_rows).  What is left adds ~1e-14 per element at
//     M = 8192 with all weights;
//   * a pass accumulates one weight over at most P pairs with
//     P (B/2)^2 M <= 2^24, so every partial sum is an integer below 2^24 and
//     the FP32 tensor-core accumulation is exact whatever its rounding mode
//     (b = 6 at M = 8192: P = 2; b = 5: P = 8);
//   * each pass's integer sums are weighted by B^-(w+2) (in FP32, exactly)
//     and added in FP64; the row and column scales multiply the sum once,
//     after the tile's last pass.
//
// Kernel layout: persistent CTAs over the 128 x 256 tiles of the upper block
// triangle, pass-major (every CTA runs pass p over its tiles before pass
// p + 1, so the CTAs stream the same two digit slices at a time and L2 holds
// their common panels); warp 0 issues TMA loads of one digit slice of the A
// rows and one of the B rows per stage (4-stage ring of 48 KB stages, 64-wide
// K blocks in 128-byte swizzled rows), warp 1 issues one MMA per 16-wide K
// step into one of two TMEM buffers (one buffer per pass, so the MMAs of the
// next pass overlap the drain of this one), warps 2-9 drain each pass into
// the FP64 output.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "gcp_device.cuh"
#include "gcp_internal.cuh"
#include "gcp_tc_ptx.cuh"

namespace gcp {

struct OzMaps {
  CUtensorMap m[kOzSlices];
};
struct OzOperands {
  OzMaps maps;
};
// The passes of one product: weight w, pairs (s, w - s) for s in
// [s0, s0 + ns).
constexpr int kOzMaxPass = 64;
struct OzPlan {
  int npass;
  int db;  // digit bits b (base B = 2^b)
  int w[kOzMaxPass];
  int s0[kOzMaxPass];
  int ns[kOzMaxPass];
};
// The slice arrays' device addresses, passed by value.
struct OzSlicePtrs {
  __half* p[kOzSlices];
};

namespace {
using namespace tcx;
// 64-wide K blocks in 128-byte swizzled rows: half as many TMA row
// requests per byte as 32-wide blocks.
constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int kThreads = 320;
constexpr uint32_t kABytes = BM * BK * 2;          // 16 KB
constexpr uint32_t kBBytes = BN * BK * 2;          // 32 KB
constexpr uint32_t kStageBytes = kABytes + kBBytes;  // 48 KB
constexpr uint32_t kTpBytes = 8 * 32 * 32 * 4;  // one 32 x 32 float block per drain warp
constexpr uint32_t kSmemBytes = STAGES * kStageBytes + kTpBytes + 1024;
static_assert(kSmemBytes + 512 <= 227 * 1024, "shared memory per CTA");
constexpr uint32_t kTmemCols = 512;

// Tile order: super-columns of 8 column blocks, row block by row block
// inside each (the tiles with I < 2J + 2), so that concurrent CTAs share
// their slice panels in L2.
__device__ __forceinline__ void oz_tile(int t, int NI, int NJ, int& I, int& J) {
  constexpr int kGroupJ = 8;
  for (int j0 = 0; j0 < NJ; j0 += kGroupJ) {
    const int j1 = j0 + kGroupJ < NJ ? j0 + kGroupJ : NJ;
    for (int i = 0; i < NI; ++i) {
      const int jstart = (i >> 1) > j0 ? (i >> 1) : j0;
      const int cnt = j1 > jstart ? j1 - jstart : 0;
      if (t < cnt) {
        I = i;
        J = jstart + t;
        return;
      }
      t -= cnt;
    }
  }
  I = 0;  // not reached for t < tc_num_tiles
  J = 0;
}

// ---- slicing ---------------------------------------------------------------
// GB300 issues FP64 at a small fraction of its integer rate, so the digits
// come from integer arithmetic: one exact power-of-two scaling and rounding
// gives the 45-bit fixed-point value n = rint(2^45 D_ij / 2^e_i), |n| <= 2^44,
// and its balanced base-32 digits follow by rounding shifts, most
// significant first, each remainder exact.
// One row i of D (the whole block works on it).
__device__ __forceinline__ void slice_row(const double* __restrict__ D, int M, int Mp, int i,
                                          int db, int nsl, __half* const* sl,
                                          double* __restrict__ rscale, __half* __restrict__ Dh,
                                          __half* __restrict__ Dl) {
  __shared__ unsigned long long red[32];
  __shared__ int e_sh;
  // row max of |D_ij| as the largest magnitude bit pattern (monotone for
  // non-negative doubles)
  unsigned long long mb = 0ull;
  if (i < M)
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
      const unsigned long long b =
          (unsigned long long)__double_as_longlong(D[(size_t)i * M + j]) & 0x7fffffffffffffffull;
      mb = b > mb ? b : mb;
    }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, mb, o);
    mb = t > mb ? t : mb;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mb;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long b = 0ull;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = red[w] > b ? red[w] : b;
    const double m = __longlong_as_double((long long)b);
    // smallest power of two with m <= 2^e / 2 (rows below 2^-900 are cut to 0)
    int e = 0;
    if (m > 0.0) {
      frexp(m, &e);  // m = f 2^e, f in [0.5, 1)
      e += 1;
    }
    e = e < -900 ? -900 : e;
    e_sh = e;
    rscale[i] = ldexp(1.0, e);
  }
  __syncthreads();
  const int nbits = db * nsl;  // fixed-point bits: |n| <= 2^(nbits - 1)
  const double to_fixed = ldexp(1.0, nbits - e_sh);  // exact: a power of two
  const float to_half = ldexpf(1.0f, 14 - nbits);
  for (int j = threadIdx.x; j < Mp; j += blockDim.x) {
    const double d = (i < M && j < M) ? D[(size_t)i * M + j] : 0.0;
    long long n = __double2ll_rn(d * to_fixed);
    const size_t o = (size_t)i * Mp + j;
    // fp16 halves of 2^14 D_ij / 2^e_i = n 2^(14 - nbits) (|.| <= 2^13), ~22 bits
    const float f = (float)n * to_half;
    const __half h = __float2half_rn(f);
    Dh[o] = h;
    Dl[o] = __float2half_rn(f - __half2float(h));
    for (int s = 0; s < nsl; ++s) {
      const int k = db * (nsl - 1 - s);
      const long long dg = k > 0 ? ((n + (1ll << (k > 0 ? k - 1 : 0))) >> k) : n;  // |dg| <= B/2
      n -= dg << k;  // exact, |n| <= 2^(k-1)
      sl[s][o] = __int2half_rn((int)dg);
    }
  }
}

__global__ void __launch_bounds__(256) oz_slice_kernel(const double* __restrict__ D, int M, int Mp,
                                                       int db, int nsl, const OzSlicePtrs slices,
                                                       double* __restrict__ rscale,
                                                       __half* __restrict__ Dh,
                                                       __half* __restrict__ Dl,
                                                       const State* __restrict__ st) {
  if (st->stopped) return;
  slice_row(D, M, Mp, blockIdx.x, db, nsl, slices.p, rscale, Dh, Dl);
}

// Batched: block (i, instance); D is the instance's current iterate.
__global__ void __launch_bounds__(256) batch_oz_slice_kernel(const BatchItem* items, int db,
                                                             int nsl) {
  const BatchItem& it = items[blockIdx.y];
  if ((int)blockIdx.x >= it.Mp || it.st->stopped) return;
  slice_row(it.D64[it.st->parity], it.M, it.Mp, blockIdx.x, db, nsl, (__half* const*)it.oz_sl,
            it.oz_rs, (__half*)it.oz_dh, (__half*)it.oz_dl);
}

// ---- finalize: traces, residual, halves of X = S - D -----------------------
// Row i of X is scaled by xscale_i = 2^(13 - e) with max_j |X_ij| < 2^e, so
// that its fp16 halves keep ~22 bits of every row whatever the size of X.
// FP64 is slow on this part, so it is kept where the arithmetic needs it:
// X = S - D (S and D are O(1), X is small), sum S o D (Tr D^3, which the
// coefficient takes differences of) and the diagonal sums.  X itself has
// 24 bits to spare in FP32, which holds the residual ||X||_F^2 (per lane,
// then FP64 across lanes), the row maximum and the halves; a thread keeps
// its first kFinCache values of the row in registers between the passes.
// The diagonal of S is replaced by sum_k D_ik^2 formed here in FP64 (a dot
// product of the row with itself, fixed reduction order), so that Tr S and
// the diagonal of X do not depend on which digit pairs the slice product
// kept (its dropped squares are all positive on the diagonal).
constexpr int kFinThreads = 256;
constexpr int kFinWarps = kFinThreads / 32;
constexpr int kFinCache = 32;  // values of a row a lane keeps: 1024 columns per warp
// One warp per row: warp w of block `blk` of `nblk` takes rows
// blk kFinWarps + w, then every nblk kFinWarps; partials into part[0..5].
__device__ __forceinline__ void finalize_rows(double* __restrict__ S,
                                              const double* __restrict__ D, int M, int Mp,
                                              int blk, int nblk, double* __restrict__ part,
                                              __half* __restrict__ Xh, __half* __restrict__ Xl,
                                              double* __restrict__ xscale) {
  __shared__ double red[32 * 5];
  const int lane = threadIdx.x & 31;
  const int gw = blk * kFinWarps + (threadIdx.x >> 5), nw = nblk * kFinWarps;
  double v0 = 0.0, v1 = 0.0, v2 = 0.0;  // Tr D, Tr S, sum S o D
  float v3 = 0.f;                       // ||S - D||_F^2
  for (int i = gw; i < Mp; i += nw) {
    float xc[kFinCache];
    float mx = 0.f;
    double sii = 0.0;  // (D^2)_ii in FP64
    if (i < M) {
      double a = 0.0;
      for (int j = lane; j < M; j += 32) {
        const double d = D[(size_t)i * M + j];
        a = fma(d, d, a);
      }
      sii = warp_sum(a);
    }
    auto element = [&](int j) -> float {
      const size_t o = (size_t)i * M + j;
      const double sv = i == j ? sii : S[o], dv = D[o];
      if (i == j) {
        S[o] = sii;
        v0 += dv;
        v1 += sv;
      }
      v2 += sv * dv;
      const float x = (float)(sv - dv);
      v3 = fmaf(x, x, v3);
      mx = fmaxf(mx, fabsf(x));
      return x;
    };
#pragma unroll
    for (int k = 0; k < kFinCache; ++k) {
      const int j = lane + 32 * k;
      xc[k] = (i < M && j < M) ? element(j) : 0.f;
    }
    if (i < M)
      for (int j = lane + 32 * kFinCache; j < M; j += 32) element(j);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);  // mx < 2^e
    const float sx = ldexpf(1.0f, 13 - e);
    if (lane == 0) xscale[i] = (double)sx;
    auto put = [&](int j, float x) {
      const float y = x * sx;  // exact: a power of two
      const __half h = __float2half_rn(y);
      Xh[(size_t)i * Mp + j] = h;
      Xl[(size_t)i * Mp + j] = __float2half_rn(y - __half2float(h));
    };
#pragma unroll
    for (int k = 0; k < kFinCache; ++k) {
      const int j = lane + 32 * k;
      if (j < Mp) put(j, xc[k]);
    }
    for (int j = lane + 32 * kFinCache; j < Mp; j += 32) {
      float x = 0.f;
      if (i < M && j < M) {
        const size_t o = (size_t)i * M + j;
        x = (float)((i == j ? sii : S[o]) - D[o]);
      }
      put(j, x);
    }
  }
  double v[5] = {v0, v1, v2, (double)v3, 0.0};
  block_sum<5>(v, red);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 5; ++k) part[k] = v[k];
    part[5] = 0.0;
  }
}

// ---- operands of the stop-test product after a refinement step ----------------
// fp16 halves of kRefScale D, of s Delta (Delta = D1 - D, |Delta| <= 1.2 R,
// s = check_delta_scale(R) puts it near 2^12, clear of the fp16 subnormals)
// and of kRefScale Delta: D Delta, Delta D and Delta (kRefScale Delta) then
// share the scale kRefScale s and one accumulator.  The last operand loses
// Delta's smallest entries to subnormals, an error of second order.
__device__ __forceinline__ void check_halves_range(
    const double* __restrict__ D, const double* __restrict__ D1, int M, int Mp,
    __half* __restrict__ Dh, __half* __restrict__ Dl, __half* __restrict__ Xh,
    __half* __restrict__ Xl, __half* __restrict__ Eh, __half* __restrict__ El,
    const State* __restrict__ st, size_t first, size_t stride) {
  const float sd = (float)check_delta_scale(st->R);  // a power of two
  const size_t n = (size_t)Mp * Mp;
  for (size_t o = first; o < n; o += stride) {
    const int i = (int)(o / Mp), j = (int)(o % Mp);
    double d = 0.0, dd = 0.0;
    if (i < M && j < M) {
      d = D[(size_t)i * M + j];
      dd = D1[(size_t)i * M + j] - d;
    }
    const float df = (float)dd;
    const float y = (float)d * (float)kRefScale, z = df * sd, w = df * (float)kRefScale;
    const __half yh = __float2half_rn(y), zh = __float2half_rn(z), wh = __float2half_rn(w);
    Dh[o] = yh;
    Dl[o] = __float2half_rn(y - __half2float(yh));
    Xh[o] = zh;
    Xl[o] = __float2half_rn(z - __half2float(zh));
    Eh[o] = wh;
    El[o] = __float2half_rn(w - __half2float(wh));
  }
}

__global__ void __launch_bounds__(256) check_halves_kernel(
    const double* __restrict__ D, const double* __restrict__ D1, int M, int Mp,
    __half* __restrict__ Dh, __half* __restrict__ Dl, __half* __restrict__ Xh,
    __half* __restrict__ Xl, __half* __restrict__ Eh, __half* __restrict__ El,
    const State* __restrict__ st) {
  if (st->stopped) return;
  check_halves_range(D, D1, M, Mp, Dh, Dl, Xh, Xl, Eh, El, st,
                     (size_t)blockIdx.x * blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
}

// Batched: block (x, instance) over the instance's Mp x Mp elements; the
// refinement step read D64[parity ^ 1] and wrote D1 = D64[parity].
__global__ void __launch_bounds__(256) batch_check_halves_kernel(const BatchItem* items) {
  const BatchItem& it = items[blockIdx.y];
  const State* st = it.st;
  if (st->stopped) return;
  const int par = st->parity;
  check_halves_range(it.D64[par ^ 1], it.D64[par], it.M, it.Mp, (__half*)it.oz_dh,
                     (__half*)it.oz_dl, (__half*)it.oz_xh, (__half*)it.oz_xl,
                     (__half*)it.oz_sl[0], (__half*)it.oz_sl[1], st,
                     (size_t)blockIdx.x * blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
}

__global__ void __launch_bounds__(kFinThreads) oz_finalize_kernel(
    double* __restrict__ S, const double* __restrict__ D, int M, int Mp,
    double* __restrict__ part, __half* __restrict__ Xh, __half* __restrict__ Xl,
    double* __restrict__ xscale, const State* __restrict__ st) {
  if (st->stopped) return;
  finalize_rows(S, D, M, Mp, blockIdx.x, gridDim.x, part + (size_t)blockIdx.x * kPartFields, Xh,
                Xl, xscale);
}

// Batched: block (b, instance), the same row partition as a single solve of
// that instance (oz_finalize_blocks(M) blocks), partials at the instance's
// slots from oz_off.
__global__ void __launch_bounds__(kFinThreads) batch_oz_finalize_kernel(const BatchItem* items,
                                                                        double* __restrict__ part) {
  const BatchItem& it = items[blockIdx.y];
  const int nblk = oz_finalize_blocks(it.M);
  if ((int)blockIdx.x >= nblk || it.st->stopped) return;
  finalize_rows(it.S64, it.D64[it.st->parity], it.M, it.Mp, blockIdx.x, nblk,
                part + (size_t)(it.oz_off + blockIdx.x) * kPartFields, (__half*)it.oz_xh,
                (__half*)it.oz_xl, it.oz_xs);
}

// ---- the exact slice GEMM ---------------------------------------------------
// One tile of the work: its block coordinates and its instance's operands.
struct OzTile {
  int I, J, M, Mp;
  const CUtensorMap* maps;
  const double* rscale;
  double* S;
  bool skip;  // batched: the instance has stopped
};

template <bool BATCHED>
__device__ __forceinline__ void oz_ctx(int t, const CUtensorMap* maps, const double* rscale,
                                       double* S, int M, int Mp, const BatchItem* items,
                                       const int* tile_inst, OzTile& c) {
  if (!BATCHED) {
    c.M = M;
    c.Mp = Mp;
    c.maps = maps;
    c.rscale = rscale;
    c.S = S;
    c.skip = false;
    oz_tile(t, Mp / BM, (Mp + BN - 1) / BN, c.I, c.J);
  } else {
    const BatchItem& it = items[tile_inst[t]];
    c.skip = it.st->stopped != 0;
    c.M = it.M;
    c.Mp = it.Mp;
    c.maps = (const CUtensorMap*)it.oz_maps;
    c.rscale = it.oz_rs;
    c.S = it.S64;
    oz_tile(t - it.tc_off, it.Mp / BM, (it.Mp + BN - 1) / BN, c.I, c.J);
  }
}

// Single solve: `maps`, `rscale`, `S`, M, Mp and `st` describe the one
// instance.  Batched: the work list `tile_inst` (the tensor-core tile list of
// the batch) names each tile's instance; every instance's operands come from
// its BatchItem, and tiles of stopped instances are skipped.
// The CTA's (pass, tile) work items in order.  Single products run pass-major
// (every tile of pass p before pass p + 1: the CTAs stream the same two
// digit slices at a time).  Batched products, whose tiles have K <= 1024 and
// whose drains' FP64 read-modify-write per pass outweighs the products, run
// tile-major: a tile's passes one after the other, so that its FP64 output
// stays in L2 between them.  Each element sums the passes in the same order
// either way.
template <bool BATCHED>
__device__ __forceinline__ void oz_work(int it, int npass, int ntl, int& ps, int& t) {
  if (BATCHED) {
    t = blockIdx.x + (it / npass) * gridDim.x;
    ps = it % npass;
  } else {
    ps = it / ntl;
    t = blockIdx.x + (it % ntl) * gridDim.x;
  }
}

template <bool BATCHED>
__global__ void __launch_bounds__(kThreads, 1)
    oz_gemm_kernel(const __grid_constant__ OzMaps maps, const __grid_constant__ OzPlan plan,
                   const double* __restrict__ rscale, double* __restrict__ S, int M, int Mp,
                   int ntiles, State* st, const BatchItem* items, const int* tile_inst) {
  if (!BATCHED && (st->stopped || st->timeout)) return;
  int* const tflag = BATCHED ? &items[0].st->timeout : &st->timeout;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t accf_bar[2];
  __shared__ __align__(8) uint64_t acce_bar[2];
  __shared__ __align__(8) uint64_t fin_bar;
  __shared__ uint32_t tmem_holder;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf_bar[b], 1);
      mbar_init(&acce_bar[b], kDrainThreads / 32);
    }
    mbar_init(&fin_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_holder)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_holder;
  // this CTA's tiles, and its (pass, tile) work items
  const int ntl = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int nwork = plan.npass * ntl;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t g = 0;
      bool alive = true;
      for (int it = 0; it < nwork && alive; ++it) {
        {
          int ps, t;
          oz_work<BATCHED>(it, plan.npass, ntl, ps, t);
          OzTile c;
          oz_ctx<BATCHED>(t, maps.m, rscale, S, M, Mp, items, tile_inst, c);
          if (c.skip) continue;
          const int nkb = c.Mp / BK;
          for (int p = plan.s0[ps]; p < plan.s0[ps] + plan.ns[ps] && alive; ++p)
            for (int kb = 0; kb < nkb; ++kb, ++g) {
              const int w = plan.w[ps];
              const uint32_t s = g % STAGES;
              if (g >= STAGES && !mbar_wait(&empty_bar[s], ((g / STAGES) - 1) & 1)) {
                atomicOr(tflag, 1);
                alive = false;
                break;
              }
              const uint32_t stage = sbase + s * kStageBytes;
              mbar_expect_tx(&full_bar[s], kStageBytes);
              const int kx = kb * BK;
              tma_load_2d(&c.maps[p], &full_bar[s], stage, kx, c.I * BM);
              tma_load_2d(&c.maps[w - p], &full_bar[s], stage + kABytes, kx, c.J * BN);
              tma_load_2d(&c.maps[w - p], &full_bar[s], stage + kABytes + kBBytes / 2, kx,
                          c.J * BN + 128);
            }
        }
      }
      const uint32_t first = g > STAGES ? g - STAGES : 0;
      for (uint32_t k = first; k < g; ++k)
        if (!mbar_wait(&full_bar[k % STAGES], (k / STAGES) & 1)) atomicOr(tflag, 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_f16(0);
      uint32_t g = 0, qc = 0;
      bool alive = true;
      for (int it = 0; it < nwork && alive; ++it) {
        {
          int ps, t;
          oz_work<BATCHED>(it, plan.npass, ntl, ps, t);
          OzTile c;
          oz_ctx<BATCHED>(t, maps.m, rscale, S, M, Mp, items, tile_inst, c);
          if (c.skip) continue;
          const int nkb = c.Mp / BK;
          const uint32_t b = qc & 1;
          if (qc >= 2 && !mbar_wait(&acce_bar[b], ((qc >> 1) - 1) & 1)) {
            atomicOr(tflag, 1);
            alive = false;
            break;
          }
          tc_fence_after();
          const uint32_t acc = tmem + b * 256;
          bool first = true;
          for (int p = plan.s0[ps]; p < plan.s0[ps] + plan.ns[ps] && alive; ++p)
            for (int kb = 0; kb < nkb; ++kb, ++g) {
              const uint32_t s = g % STAGES;
              if (!mbar_wait(&full_bar[s], (g / STAGES) & 1)) {
                atomicOr(tflag, 1);
                alive = false;
                break;
              }
              tc_fence_after();
              const uint32_t a = sbase + s * kStageBytes;
              const uint32_t bb = a + kABytes;
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) {
                const uint32_t off = kk * 32;
                umma(acc, sdesc128(a + off), sdesc128(bb + off), idesc, first ? 0u : 1u);
                first = false;
              }
              umma_commit(&empty_bar[s]);
            }
          umma_commit(&accf_bar[b]);
          ++qc;
        }
      }
      umma_commit(&fin_bar);
      if (!mbar_wait(&fin_bar, 0)) atomicOr(tflag, 1);
    }
  } else {
    const int dw = warp - 2, q = warp & 3, half = dw >> 2;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    float* tp = reinterpret_cast<float*>(smem_raw + (sbase - raw) + STAGES * kStageBytes) +
                dw * 32 * 32;
    uint32_t qc = 0;
    bool alive = true;
    for (int it = 0; it < nwork && alive; ++it) {
      int ps, t;
      oz_work<BATCHED>(it, plan.npass, ntl, ps, t);
      // B^-(w+2), applied in FP32: the pass sums are integers below 2^24, so
      // the product is exact (B^-(w+2) >= 2^-60 stays normal)
      const float wscale = ldexpf(1.0f, -plan.db * (plan.w[ps] + 2));
      const bool first_pass = ps == 0, last_pass = ps == plan.npass - 1;
      {
        OzTile c;
        oz_ctx<BATCHED>(t, maps.m, rscale, S, M, Mp, items, tile_inst, c);
        if (c.skip) continue;
        const int Mi = c.M;
        double* const Si = c.S;
        const int row = c.I * BM + 32 * q + lane;
        const int jb = 2 * c.J + half, c_base = c.J * BN + half * 128;
        const bool need = jb >= c.I, diag = jb == c.I;
        const double rs_row = row < Mi ? c.rscale[row] : 0.0;
        const uint32_t b = qc & 1;
        const bool got = __all_sync(0xffffffffu, mbar_wait(&accf_bar[b], (qc >> 1) & 1));
        if (!got) {
          if (lane == 0) atomicOr(tflag, 1);
          alive = false;
          break;
        }
        tc_fence_after();
        const uint32_t base = tmem + lane_base + b * 256 + half * 128;
        const int row0 = c.I * BM + 32 * q;
#pragma unroll 1
        for (int part = 0; part < 4; ++part) {
          uint32_t r[32];
          tmem_ld32(base + part * 32, r);
          tmem_ld_wait();
          if (!need) continue;  // warp-uniform
          // transpose the 32 x 32 block through shared memory (XOR-swizzled,
          // conflict-free): lane = row -> lane = column, so that the FP64
          // read-modify-write below is one 256-byte segment per row
#pragma unroll
          for (int k = 0; k < 32; ++k) tp[lane * 32 + (k ^ lane)] = __uint_as_float(r[k]);
          __syncwarp();
          float a[32];
#pragma unroll
          for (int k = 0; k < 32; ++k) a[k] = tp[k * 32 + (lane ^ k)];
          __syncwarp();
          const int cc = c_base + part * 32 + lane;
          // the row and column scales 2^(e_i + e_j) multiply the tile once,
          // on its last pass: the passes add unscaled terms, and power-of-
          // two scaling commutes with the rounding of the FP64 additions
          // (the result equals scaling every term, short of underflow)
          const double cs = (last_pass && cc < Mi) ? c.rscale[cc] : 0.0;
          double old[32];
          if (!first_pass) {
#pragma unroll
            for (int k = 0; k < 32; ++k) {
              const int rk = row0 + k;
              const bool ok = rk < Mi && cc < Mi && !(diag && cc < rk);
              old[k] = ok ? Si[(size_t)rk * Mi + cc] : 0.0;
            }
          }
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            const int rk = row0 + k;
            const bool ok = rk < Mi && cc < Mi && !(diag && cc < rk);
            const double v = (double)(a[k] * wscale);  // exact
            double x = first_pass ? v : old[k] + v;
            if (last_pass) x *= cs * __shfl_sync(0xffffffffu, rs_row, k);
            if (ok) Si[(size_t)rk * Mi + cc] = x;
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce_bar[b]);
        ++qc;
        // mirror the finished tile (values stored by other lanes of this warp)
        __syncwarp();
        if (last_pass && need && row < Mi) {
          for (int k = 0; k < 128; ++k) {
            const int col = c_base + k;
            if (col >= Mi || (diag && col <= row)) continue;
            Si[(size_t)col * Mi + row] = Si[(size_t)row * Mi + col];
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols));
  }
}

int sm_count() {
  static int n = 0;
  if (n > 0) return n;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
    n = 148;
  return n;
}
}  // namespace

int oz_make_operands(OzOperands** op, void* const* slices, int Mp, char* err, int errlen) {
  OzOperands* o = new OzOperands;
  for (int s = 0; s < kOzSlices; ++s)
    if (tc_encode_map(&o->maps.m[s], slices[s], Mp, 0, err, errlen, BK)) {
      delete o;
      return 1;
    }
  *op = o;
  return 0;
}

void oz_free_operands(OzOperands* op) { delete op; }

void launch_oz_slice(const double* D, int M, int Mp, void* const* slices, double* rscale,
                     void* Dh, void* Dl, const State* st, cudaStream_t s) {
  OzSlicePtrs sp;
  for (int k = 0; k < kOzSlices; ++k) sp.p[k] = (__half*)slices[k];
  oz_slice_kernel<<<Mp, 256, 0, s>>>(D, M, Mp, oz_digit_bits(M), oz_num_slices(M), sp, rscale,
                                     (__half*)Dh, (__half*)Dl, st);
}

// Digit width of the slicing for an M-long inner dimension: 6 bits (8
// slices) while a pass can hold a pair, (B/2)^2 M <= 2^24, else 5 (9 slices).
int oz_digit_bits(int M) { return M <= 16384 ? 6 : 5; }
int oz_num_slices(int M) { return oz_digit_bits(M) == 6 ? 8 : 9; }

// Highest weight a refinement step with stop tolerance tol keeps.  Dropping
// the weights above W leaves, per element of D^2, the sum over k of the
// pair terms of weight W + 1: with row scales 2^e <= 1 (|D_ij| <= 1/2 for a
// near-idempotent D), digits of mean square (B/2)^2 / 3 and independent
// signs, its size is ~ (B/2)^2/3 B^-(W+3) sqrt(M n_{W+1}) (n_w pairs of
// weight w), and over the M^2 elements
//   F(W) = (B/2)^2 / 3  B^-(W+3)  M^1.5  sqrt(n_{W+1})
// in the Frobenius norm, which adds to ||D^2 - D||_F after the step (the
// residuals measured against a host FP64 recomputation at M = 257..2048
// stayed 2-20x below it).  F is taken at the largest M of the digit base
// (16384 for b = 6, 32768 for b = 5), so that W depends on tol alone and a
// batch shares the plan of its single solves; W is the smallest weight with
// F(W) <= tol / 8: tol = 1e-6 gives W = 6 (28 products instead of 43;
// F = 1.1e-7), tol = 1e-7 W = 7 (36), tol <= 1e-8 all weights (43).  The
// diagonal of D^2, whose dropped squares do not cancel, is formed exactly in
// FP64 whatever W (finalize_rows), so Tr D^2 does not depend on it; the
// idempotency stop test compares the
// residual with tol - F(W) (oz_tail_estimate), so that the residual of the
// exact square of the returned D stays below tol.
namespace {
double oz_tail(int db, int W) {
  const int nsl = db == 6 ? 8 : 9;
  const double B = (double)(1 << db), h = B / 2.0, Mref = db == 6 ? 16384.0 : 32768.0;
  const int lo = (W + 1) - (nsl - 1) > 0 ? (W + 1) - (nsl - 1) : 0;
  const int hi = W + 1 < nsl - 1 ? W + 1 : nsl - 1;
  const double np = hi >= lo ? (double)(hi - lo + 1) : 0.0;
  return h * h / 3.0 * pow(B, -(double)(W + 3)) * pow(Mref, 1.5) * sqrt(np);
}
}  // namespace

int oz_weight_cap(int M, double tol) {
  const int db = oz_digit_bits(M), nsl = oz_num_slices(M);
  for (int W = 2; W < nsl; ++W)
    if (oz_tail(db, W) <= tol / 8.0) return W;
  return nsl;
}

double oz_tail_estimate(int M, double tol) {
  const int db = oz_digit_bits(M), W = oz_weight_cap(M, tol);
  if (W >= oz_num_slices(M)) return 0.0;  // all weights: the plan's floor is ~1e-14 M
  return oz_tail(db, W);
}

namespace {
// Passes for an M-long inner dimension: pairs (s, w - s) with
// 0 <= s, w - s < ns for the kept weights w <= wcap (at most b = 6: 0..8;
// b = 5: 0..9), at most floor(2^24 / ((B/2)^2 M)) pairs a pass.
int oz_plan(int M, int wcap, OzPlan* plan) {
  const int db = oz_digit_bits(M), nsl = oz_num_slices(M);
  const int wmax = (wcap > 0 && wcap < nsl) ? wcap : nsl;  // 8 (b = 6) or 9 (b = 5) at most
  const long long half = 1ll << (db - 1);
  const long long cap = (1ll << 24) / (half * half * M);
  if (cap < 1) return 1;
  plan->npass = 0;
  plan->db = db;
  for (int w = 0; w <= wmax; ++w) {
    int lo = w - (nsl - 1) > 0 ? w - (nsl - 1) : 0;
    const int hi = w < nsl - 1 ? w : nsl - 1;
    while (lo <= hi) {
      const int n = (hi - lo + 1) < cap ? (hi - lo + 1) : (int)cap;
      if (plan->npass >= kOzMaxPass) return 1;
      plan->w[plan->npass] = w;
      plan->s0[plan->npass] = lo;
      plan->ns[plan->npass] = n;
      ++plan->npass;
      lo += n;
    }
  }
  return 0;
}
}  // namespace

int oz_num_products(int M, int wcap) {
  OzPlan plan;
  if (oz_plan(M, wcap, &plan)) return 0;
  int n = 0;
  for (int p = 0; p < plan.npass; ++p) n += plan.ns[p];
  return n;
}

int launch_oz_gemm(const OzOperands* op, const double* rscale, double* S64, int M, int Mp,
                   int wcap, State* st, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(oz_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSmemBytes) != cudaSuccess)
      return 1;
    attr = true;
  }
  const int ntiles = tc_num_tiles(Mp);
  const int grid = ntiles < sm_count() ? ntiles : sm_count();
  OzPlan plan;
  if (oz_plan(M, wcap, &plan)) return 1;
  oz_gemm_kernel<false><<<grid, kThreads, kSmemBytes, s>>>(op->maps, plan, rscale, S64, M, Mp,
                                                           ntiles, st, nullptr, nullptr);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 1;
}

int launch_batch_oz_gemm(const BatchItem* items, const int* tile_inst, int ntiles, int maxM,
                         int wcap, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(oz_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSmemBytes) != cudaSuccess)
      return 1;
    attr = true;
  }
  const int grid = ntiles < sm_count() ? ntiles : sm_count();
  // the pass plan of the largest instance is valid for every smaller one
  // (and equal to theirs up to M = 7281, where every weight fits one pass)
  OzPlan plan;
  if (oz_plan(maxM, wcap, &plan)) return 1;
  OzMaps none;
  memset(&none, 0, sizeof none);
  oz_gemm_kernel<true><<<grid, kThreads, kSmemBytes, s>>>(none, plan, nullptr, nullptr, 0, 0,
                                                          ntiles, nullptr, items, tile_inst);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 1;
}

void launch_batch_oz_slice(const BatchItem* items, int batch, int maxM, cudaStream_t s) {
  const int maxMp = tc_pad(maxM);
  dim3 g(maxMp, batch);
  // every instance is sliced like the largest, whose pass plan all share
  batch_oz_slice_kernel<<<g, 256, 0, s>>>(items, oz_digit_bits(maxM), oz_num_slices(maxM));
}

void launch_batch_oz_finalize(const BatchItem* items, int batch, int maxM, double* part,
                              cudaStream_t s) {
  dim3 g(oz_finalize_blocks(maxM), batch);
  batch_oz_finalize_kernel<<<g, kFinThreads, 0, s>>>(items, part);
}

size_t oz_batch_map_bytes() { return (kOzSlices + 6) * sizeof(CUtensorMap); }

int oz_build_batch_maps(void* maps_host, const BatchItem& it, char* err, int errlen) {
  CUtensorMap* m = (CUtensorMap*)maps_host;
  for (int k = 0; k < kOzSlices; ++k)
    if (tc_encode_map(&m[k], it.oz_sl[k], it.Mp, 0, err, errlen, BK)) return 1;
  const void* halves[6] = {it.oz_dh, it.oz_dl, it.oz_xh, it.oz_xl, it.oz_sl[0], it.oz_sl[1]};
  for (int k = 0; k < 6; ++k)
    if (tc_encode_map(&m[kOzSlices + k], halves[k], it.Mp, 0, err, errlen)) return 1;
  return 0;
}


void launch_check_halves(const double* D64, const double* D1, int M, int Mp, void* Dh, void* Dl,
                         void* Xh, void* Xl, void* Eh, void* El, const State* st,
                         cudaStream_t s) {
  const size_t n = (size_t)Mp * Mp;
  const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  check_halves_kernel<<<grid, 256, 0, s>>>(D64, D1, M, Mp, (__half*)Dh, (__half*)Dl, (__half*)Xh,
                                           (__half*)Xl, (__half*)Eh, (__half*)El, st);
}

void launch_batch_check_halves(const BatchItem* items, int batch, int maxM, cudaStream_t s) {
  const long long n = (long long)tc_pad(maxM) * tc_pad(maxM);
  long long b = (n + 8191) / 8192;  // ~32 elements a thread for the largest instance
  b = b < 1 ? 1 : (b > 64 ? 64 : b);
  batch_check_halves_kernel<<<dim3((unsigned)b, batch), 256, 0, s>>>(items);
}

void launch_oz_finalize(double* S64, const double* D64, int M, int Mp, double* part,
                        void* Xh, void* Xl, double* xscale, const State* st, cudaStream_t s) {
  oz_finalize_kernel<<<oz_finalize_blocks(M), kFinThreads, 0, s>>>(
      S64, D64, M, Mp, part, (__half*)Xh, (__half*)Xl, xscale, st);
}

}  // namespace gcp
