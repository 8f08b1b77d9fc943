// Split-precision tensor-core products of one GCP step (sm_103a: tcgen05 +
// TMEM + TMA), with the step's elementwise work fused into the epilogues:
// mode 1 GEMM1, mode 2 GEMM2 of the split phase; mode 3 the product of an
// exact-slice refinement step, mode 4 the stop-test product after it
// (W = D1^2 - D^2 over a K = 3M concatenation of operands); modes 5 and 6
// plain products C = A B (FP32 out) for the adjoint, over all tiles (mode 5,
// a non-symmetric result) or the upper tiles mirrored (mode 6).
//
// State.  The iterate is held shifted, X = D - theta J (J = identity on the
// unpadded M x M block), in FP32, plus two 16-bit halves of s X (s = 2^14):
// h = rn(sX), l = rn(sX - h).  Early in the recursion D is close to
// theta I, so X is small and the rounding of the state and of the products
// is relative to |X|, not to |D|: the shift costs nothing (Tr D = N fixes
// theta) and keeps the subspace of the final projector from being rotated by
// rounding while the occupied and virtual eigenvalues of D are still close.
//
// Products.  A B^T with both operands K-major; every operand is symmetric,
// so B = B^T.  Per K step three MMAs (Ah Bh, Ah Bl, Al Bh) accumulate into
// one TMEM accumulator (the lo*lo term is below FP32 resolution).
//
// Accumulation.  The tensor cores add each MMA (K = 16) into their FP32
// accumulator with truncation (round toward zero), so the error of a product
// comes from the MMAs that round at the scale of the accumulated sum, and it
// rotates the occupied subspace of the final D (noise that does not commute
// with D is never purified away).  Two measures:
//   * the accumulator holds one K chunk only (128 for the split products, 32
//     for the refinement product, whose trace must hold to ~1e-10): eight
//     drain warps add each chunk into FP32 registers with round-to-nearest
//     while the MMA warp fills the other of two TMEM buffers (over all of
//     K = 8192 the truncation biased same-sign sums by ~6e-5 relative;
//     shorter chunks only trade it for more register adds: 64 and 32 gave
//     1.13e-6 and 1.49e-6 against 9.9e-7 for the subspace error of the
//     M = 8192 solve);
//   * inside a chunk the two cross products (hi x lo, lo x hi: 2^-11 of the
//     result) are issued first, so they round at their own scale, and only
//     the hi x hi MMAs round at the scale of the result (one per K step
//     instead of three): 8.4e-7 against 9.9e-7 at M = 8192.  Both GEMMs of
//     a step must use the same order (either one alone measured worse than
//     neither).  A chunk's stages stay resident until its hi x hi pass, so
//     each stage has separate barriers for its hi and lo halves: the lo
//     halves are released after the cross pass and refilled early, and only
//     the hi halves wait for the end of the chunk.
//
// GEMM1 (Y = X X).  With S = D^2 = theta^2 J + Sigma, Sigma = 2 theta X + Y,
// the epilogue writes Sigma (FP32 + halves, exactly symmetric) and per-tile
// partial sums Tr X, Tr Sigma, sum Sigma o X, ||S - D||_F^2 (elementwise,
// S - D = Sigma - X - theta(1-theta) J) and optionally sum D o H, from which
// the control kernel forms Tr D, Tr D^2, Tr D^3 (Eq. mcwgamb).
// GEMM2 (Z = X Sigma).  D_{n+1} = a D + b S + g3 D S (HPCP, Eq. hpcp3:
// a = 1 - 2c, b = 2 + 2c, g3 = -2; PMCP, Eq. pm1, other coefficients)
// becomes, for X_{n+1} = D_{n+1} - theta J, with D S = theta^3 J +
// theta^2 X + theta Sigma + Z,
//   X_{n+1} = xshift J + (a + g3 theta^2) X + (b + g3 theta) Sigma + g3 Z,
//   xshift = a theta + b theta^2 + g3 theta^3 - theta
//          (= 2 theta (1-theta)(theta - c) for HPCP).
//
// Schedule.  Persistent CTAs (one per SM) walk the 128 x 256 tiles of the
// upper block triangle with four warpgroups of specialised warps:
//   * warpgroup 0: warp 0 lane 0 issues the TMA loads (SWIZZLE_64B, 32-wide
//     K blocks; each stage's hi part and lo part, 24 KB each, in rings of 5
//     and 4 slots), warp 1 lane 0 the tcgen05.mma;
//   * warpgroups 1-2, eight drain warps: warp w reads TMEM lanes
//     32 (w % 4).. and columns 128 ((w - 4) / 4).. of each chunk and keeps
//     the tile's 128 x 256 FP32 sum in registers (128 a thread); at the end
//     of a tile they store it to one of two scratch slots of this CTA in
//     global memory (128 KB each, L2-resident) and start on the next tile
//     (a non-symmetric plain product, mode 5, they store scaled themselves);
//   * warpgroup 3, four epilogue warps: the tile's epilogue from the scratch
//     slot while the next tile accumulates, its 32 x 32 blocks dealt
//     round-robin to the four warps; each warp mirrors its blocks through a
//     16 x 32 shared-memory buffer and, in batched launches, prefetches into
//     L2 the rows of the next tile that it will read from HBM.
// So the MMA warp never waits for an epilogue (it waited ~25 % of a tile at
// M = 8192 when the drain warps also ran the epilogue).  Register budgets
// (setmaxnreg): 40 / 176 / 120 a thread against 128 at launch (40 / 168 /
// 136 in the batched kernels).  Blocks
// below the diagonal are skipped; every element above the diagonal is
// stored twice (direct and mirrored).  Every wait is bounded (2 s unless the
// launch asks for less); on expiry the kernel records State::timeout and
// winds down, still freeing its TMEM.
#include <cuda.h>
#include <stdio.h>
#include <string.h>

#include "gcp_device.cuh"
#include "gcp_internal.cuh"
#include "gcp_tc_ptx.cuh"

namespace gcp {

struct TcOperands {
  CUtensorMap hi;
  CUtensorMap lo;
};

namespace {
using namespace tcx;
constexpr int BM = 128, BN = 256, BK = 32;
// Operand ring: every 32-wide K block ("stage") has a hi part (A hi, B hi)
// and a lo part (A lo, B lo) of 24 KB each, in separate rings.  The cross
// products of a chunk read both, the hi x hi pass at its end only the hi
// part, so the hi ring has one slot more: the next chunk's first hi part
// loads while the current chunk is still in its cross pass.
constexpr int kLoSlots = 4, kHiSlots = 5;
// K chunk per TMEM drain, in 32-wide K blocks (see the header comment).
template <int MODE>
__host__ __device__ constexpr int kc_stages() {
  return MODE == 3 ? 1 : 4;
}
static_assert(4 <= kLoSlots && 4 < kHiSlots, "a chunk must fit the rings");
constexpr int kThreads = 512;
constexpr int kEpiWarp0 = 12;  // first epilogue warp
constexpr int kEpiThreads = 128;
constexpr int kEpiBarrier = 2;  // named barrier of the epilogue warps
// Register split (setmaxnreg, per thread) against 128 a thread at launch:
// the batched kernels, whose short-K tiles leave the drain warps idle and
// the epilogue warps busy, move 8 registers a drain thread to the epilogue
// (136, so a 32 x 32 block's loads are all in flight at once without
// spilling).
constexpr uint32_t kCtlRegs = 40;
template <bool BATCHED>
__host__ __device__ constexpr uint32_t drain_regs() { return BATCHED ? 168 : 176; }
template <bool BATCHED>
__host__ __device__ constexpr uint32_t epi_regs() { return BATCHED ? 136 : 120; }
template <bool BATCHED>
__host__ __device__ constexpr uint32_t split_regs() {
  return 128 * kCtlRegs + 256 * drain_regs<BATCHED>() + 128 * epi_regs<BATCHED>();
}
static_assert(split_regs<false>() <= 65536 && split_regs<true>() <= 65536, "register split");
constexpr uint32_t kABytes = BM * BK * 2;           // 8 KB
constexpr uint32_t kBBytes = BN * BK * 2;           // 16 KB
constexpr uint32_t kPartBytes = kABytes + kBBytes;  // 24 KB: the hi (or lo) part of a stage
constexpr uint32_t kSmemBytes = (kLoSlots + kHiSlots) * kPartBytes + 1024;
static_assert(kSmemBytes + 1024 <= 227 * 1024, "shared memory per CTA");
constexpr uint32_t kTmemCols = 512;  // two 256-column accumulator buffers
// Scratch slot: a finished tile, row-major (BM x BN).
constexpr size_t kTileFloats = (size_t)BM * BN;
constexpr size_t kSlotFloats = kTileFloats;  // one row-major tile per scratch slot

struct Epi {
  const float* X;    // current shifted iterate (FP32, Mp x Mp)
  const float* Sig;  // Sigma (mode 2)
  float* out;        // Sigma (mode 1) or X_{n+1} (mode 2), FP32
  void* out_h;       // split halves of `out`
  void* out_l;
  const void* H;     // optional, for sum D o H (mode 1)
  int h_f64, ldh;
  double* part;      // per-tile partials (modes 1 and 4)
  State* st;
  int M, Mp, ntiles;
  float split_scale;  // s
  float inv_s2;       // 1/s^2
  // mode 3 (McWeeny refinement in FP64): D+ = S - 2 Z - a (S - D),
  // Z = (S - D) D, a = 1 - 2c from the state
  const double* S64;
  const double* D64;
  double* Dn64;
  const double* rs_x;  // row scales of the X operand
  const double* rs_d;  // 2^e_j: row j of the D operand holds kRefScale D_jk / 2^e_j
  int ld64;
  // mode 4 (stop test after a refinement step): S64 = D^2 (exact), D64 = the
  // new iterate D1, the product W = D1^2 - D^2 in the scale kRefScale s_Delta;
  // emaps: device maps of Delta at the scale kRefScale (B of the Delta^2 part)
  const CUtensorMap* emaps;
  // drain -> epilogue hand-over: 2 slots of BM x BN floats per CTA
  float* scratch;
  // batched: the order in which the CTAs take the tiles (position -> tile
  // id of the work list), or null for the work list's own order; a tile's
  // partials stay at its id
  const int* order;
  unsigned long long wait_ns;  // bound of every wait
  int stall;  // diagnostic: the drain first waits on a barrier nobody arrives on
};

// Linear tile index -> (I, J): I a 128-row block, J a 256-column block,
// kept when the tile reaches the upper block triangle (I < 2J + 2, i.e.
// J >= floor(I / 2)).  Order: super-columns of kGroupJ column blocks; in
// each, row block by row block, the super-column's tiles of that row.  The
// CTAs working at the same time then share a few A panels (rows) and the
// super-column's B panels, which stay in L2 while the CTAs stream along K.
constexpr int kGroupJ = 8;
// Column blocks of 256 over an Mp x Mp operand (Mp a multiple of 128): the
// last one reaches past the matrix by 128 columns when Mp / 128 is odd; its
// B rows there load as zeros (TMA fill) and its blocks there are not stored.
__host__ __device__ __forceinline__ int nj_blocks(int Mp) { return (Mp + BN - 1) / BN; }
__host__ __device__ __forceinline__ void tc_tile(int t, int NI, int NJ, int& I, int& J) {
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

__device__ __forceinline__ void load_row32(const float* __restrict__ src, float (&a)[32]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(src) + k);
    a[4 * k] = v.x;
    a[4 * k + 1] = v.y;
    a[4 * k + 2] = v.z;
    a[4 * k + 3] = v.w;
  }
}

// All tiles (mode 5, a non-symmetric product), in the same super-column
// order: t -> (I, J) with I in [0, NI), J in [0, NJ).
__device__ __forceinline__ void tc_tile_full(int t, int NI, int NJ, int& I, int& J) {
  const int per = NI * kGroupJ;  // tiles of one full super-column
  const int j0 = (t / per) * kGroupJ;
  const int w = (NJ - j0) < kGroupJ ? (NJ - j0) : kGroupJ;
  const int r = t - (t / per) * per;
  I = r / w;
  J = j0 + r % w;
}

// Refinement-product epilogue of one thread: its row, 32 columns c_base..,
// acc[] = (A B)_row,c in the slice scale, read from the scratch row `src`.
// McWeeny refinement step in FP64 (Eq. mcweeny3): with S = D^2 exact and
// X = S - D small, 3D^2 - 2D^3 = S - 2 X D; the product Z = X D only needs
// the relative accuracy of the split product because |X| is small.  The
// general step of Eq. hpcp3 is the same plus (1 - 2c)(D - S); the control
// kernel sets c within 1/2 +- 0.05 to put Tr D+ back at N.
// Columns whose FP64 operands a refinement or stop-test thread loads at once.
constexpr int kSegGroup = 4;

__device__ __forceinline__ void refine_seg(const Epi& ep, int row, int c_base, bool diag_blk,
                                           const float* __restrict__ src) {
  if (row >= ep.M) return;
  float acc[32];
  load_row32(src, acc);
  const double wr = 1.0 / (kRefScale * ep.rs_x[row]);  // powers of two: exact
  const double g = ep.st->a;
  // a group of columns' loads in flight before their stores
#pragma unroll
  for (int k0 = 0; k0 < 32; k0 += kSegGroup) {
    double sv[kSegGroup], dv[kSegGroup], rd[kSegGroup];
#pragma unroll
    for (int j = 0; j < kSegGroup; ++j) {
      const int c = c_base + k0 + j;
      const bool ok = c < ep.M && !(diag_blk && c < row);
      const size_t o = (size_t)row * ep.ld64 + c;
      sv[j] = ok ? ep.S64[o] : 0.0;
      dv[j] = ok ? ep.D64[o] : 0.0;
      rd[j] = ok ? ep.rs_d[c] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < kSegGroup; ++j) {
      const int c = c_base + k0 + j;
      if (c >= ep.M || (diag_blk && c < row)) continue;
      const size_t o = (size_t)row * ep.ld64 + c;
      const double v = sv[j] - 2.0 * (wr * rd[j]) * (double)acc[k0 + j] - g * (sv[j] - dv[j]);
      ep.Dn64[o] = v;
      if (c != row) ep.Dn64[(size_t)c * ep.ld64 + row] = v;
    }
  }
}

// Stop-test epilogue of one thread after a refinement step D -> D1 (mode 4):
// acc[] = kRefScale s_Delta W_row,c with W = D1^2 - D^2 = D Delta + Delta D +
// Delta^2, Delta = D1 - D; with S = D^2 exact, D1^2 - D1 = S + W - D1 is
// formed in FP64 (S and D1 are O(1), the result is ~R1).  Sums: the
// residual R1^2 (FP32 per lane, weight 2 above the diagonal), Tr D1 and
// Tr D1^2 = Tr S + Tr W (FP64, diagonal only).
__device__ __forceinline__ void check_seg(const Epi& ep, int row, int c_base, bool diag_blk,
                                          const float* __restrict__ src, float inv_scale,
                                          float (&pp)[3], double (&dpart)[2]) {
  if (row >= ep.M) return;
  float acc[32];
  load_row32(src, acc);
  // a group of columns' loads in flight at a time
#pragma unroll
  for (int k0 = 0; k0 < 32; k0 += kSegGroup) {
    double sv[kSegGroup], dv[kSegGroup];
#pragma unroll
    for (int j = 0; j < kSegGroup; ++j) {
      const int c = c_base + k0 + j;
      const bool ok = c < ep.M && !(diag_blk && c < row);
      const size_t o = (size_t)row * ep.ld64 + c;
      sv[j] = ok ? ep.S64[o] : 0.0;
      dv[j] = ok ? ep.D64[o] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < kSegGroup; ++j) {
      const int k = k0 + j;
      const int c = c_base + k;
      if (c >= ep.M || (diag_blk && c < row)) continue;
      const double sw = sv[j] + (double)(acc[k] * inv_scale);  // D1^2, exact scaling
      const double d1 = dv[j];
      const float x1 = (float)(sw - d1);
      pp[1] = fmaf((c == row ? 1.f : 2.f) * x1, x1, pp[1]);
      if (c == row) {
        dpart[0] += d1;
        dpart[1] += sw;
      }
    }
  }
}

template <bool BF16>
__device__ __forceinline__ void store_out4(const Epi& ep, size_t off, float4 o) {
  using HT = typename Split<BF16>::T;
  HT h[4], l[4];
  Split<BF16>::split(o.x * ep.split_scale, h[0], l[0]);
  Split<BF16>::split(o.y * ep.split_scale, h[1], l[1]);
  Split<BF16>::split(o.z * ep.split_scale, h[2], l[2]);
  Split<BF16>::split(o.w * ep.split_scale, h[3], l[3]);
  *reinterpret_cast<float4*>(ep.out + off) = o;
  *reinterpret_cast<uint2*>(reinterpret_cast<HT*>(ep.out_h) + off) = *reinterpret_cast<uint2*>(h);
  *reinterpret_cast<uint2*>(reinterpret_cast<HT*>(ep.out_l) + off) = *reinterpret_cast<uint2*>(l);
}

template <bool BF16>
__device__ __forceinline__ void store_out1(const Epi& ep, size_t off, float o) {
  using HT = typename Split<BF16>::T;
  HT h, l;
  Split<BF16>::split(o * ep.split_scale, h, l);
  ep.out[off] = o;
  reinterpret_cast<HT*>(ep.out_h)[off] = h;
  reinterpret_cast<HT*>(ep.out_l)[off] = l;
}

// The epilogues of the split GEMMs work on 32 x 32 blocks of the output with
// eight lanes per row and four consecutive columns per lane, so every load
// and store is a whole 128-byte row segment.  A block above the diagonal is
// written twice: the direct pass (rows r, columns c) computes it from the
// row-major scratch tile and stores it; each 16-row half of its values then
// goes through a per-warp shared-memory buffer and is stored transposed
// (rows c, columns r), so the mirror costs no loads.  On a diagonal block
// the direct pass keeps the elements on or above the diagonal and the
// mirror those strictly below.
constexpr int kStageLd = 33;  // row stride of a warp's 16 x 32 staging buffer (floats)
constexpr int kStageFloats = 16 * kStageLd;

// Transposed store of the 16 x 32 values in `stage` (rows h16.. of the
// direct block with first row orow0 and first column ocol0): output rows
// ocol0 + c, columns orow0 + h16 + r; on a diagonal block only the elements
// below the diagonal.  put4(off, float4) / put1(off, float) store.
template <typename Put4, typename Put1>
__device__ __forceinline__ void mirror_half(const float* __restrict__ stage, int Mp, int orow0,
                                            int ocol0, int h16, bool diag_blk, Put4 put4,
                                            Put1 put1) {
  const int lane = threadIdx.x & 31;
  const int mc = 4 * (lane & 3);
#pragma unroll 1
  for (int k = 0; k < 4; ++k) {
    const int mr = (lane >> 2) + 8 * k;
    const float4 o = make_float4(stage[(mc + 0) * kStageLd + mr], stage[(mc + 1) * kStageLd + mr],
                                 stage[(mc + 2) * kStageLd + mr], stage[(mc + 3) * kStageLd + mr]);
    const int R = ocol0 + mr, C = orow0 + h16 + mc;
    const size_t off = (size_t)R * Mp + C;
    if (!diag_blk) {
      put4(off, o);
    } else {
      const float ov[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (C + q < R) put1(off + q, ov[q]);
    }
  }
}

// GEMM1 epilogue of one warp for one 32 x 32 block and its mirror: output
// rows orow0.., columns ocol0..; `yb` points at s^2 (X X) for the block's
// first element in the scratch tile, row stride ys.  Sigma = 2 theta X + Y
// and its halves are stored, and the partial sums accumulated.
template <bool BF16>
__device__ __forceinline__ void gemm1_pass(const Epi& ep, const float* __restrict__ yb, int ys,
                                           int orow0, int ocol0, bool diag_blk, float thf,
                                           float f2th, float thtb, float (&pp)[3],
                                           double (&dpart)[2], float* __restrict__ stage) {
  const int lane = threadIdx.x & 31;
  const int Mp = ep.Mp;
  const float is2 = ep.inv_s2;
  const int rs = lane >> 3, cl = 4 * (lane & 7);
  const size_t cbase = (size_t)ocol0 + cl;
  // the whole block's loads in flight before its first store
  float4 xv[8], yv[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int rr = rs + 4 * j;
    xv[j] = *reinterpret_cast<const float4*>(ep.X + (size_t)(orow0 + rr) * Mp + cbase);
    yv[j] = __ldcg(reinterpret_cast<const float4*>(yb + rr * ys + cl));
  }
#pragma unroll
  for (int jh = 0; jh < 8; jh += 4) {
    const float4* xx = xv + jh;
    const float4* yy = yv + jh;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = orow0 + rs + 4 * (jh + j);
      const size_t off = (size_t)r * Mp + cbase;
      float4 o;
      o.x = fmaf(f2th, xx[j].x, yy[j].x * is2);  // Sigma = 2 theta X + Y
      o.y = fmaf(f2th, xx[j].y, yy[j].y * is2);
      o.z = fmaf(f2th, xx[j].z, yy[j].z * is2);
      o.w = fmaf(f2th, xx[j].w, yy[j].w * is2);
      {
        float* st = stage + (rs + 4 * j) * kStageLd + cl;
        st[0] = o.x;
        st[1] = o.y;
        st[2] = o.z;
        st[3] = o.w;
      }
      if (!diag_blk) {
        // every element lies above the diagonal (weight 2: it stands for
        // its mirror too)
        const float ex = o.x - xx[j].x, ey = o.y - xx[j].y, ez = o.z - xx[j].z,
                    ew = o.w - xx[j].w;
        pp[0] += 2.f * (o.x * xx[j].x + o.y * xx[j].y + o.z * xx[j].z + o.w * xx[j].w);
        pp[1] += 2.f * (ex * ex + ey * ey + ez * ez + ew * ew);
        store_out4<BF16>(ep, off, o);
      } else {
        const float xs[4] = {xx[j].x, xx[j].y, xx[j].z, xx[j].w};
        const float os[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int c = ocol0 + cl + i;
          if (c < r) continue;
          const bool on_diag = c == r && r < ep.M;
          const float w = c == r ? 1.f : 2.f;
          const float e = os[i] - xs[i] - (on_diag ? thtb : 0.f);  // (S - D)_rc
          pp[0] += w * os[i] * xs[i];
          pp[1] += w * e * e;
          if (on_diag) {
            dpart[0] += (double)xs[i];
            dpart[1] += (double)os[i];
          }
          store_out1<BF16>(ep, off + i, os[i]);
        }
      }
      if (ep.H) {
        const float xs[4] = {xx[j].x, xx[j].y, xx[j].z, xx[j].w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int cc = ocol0 + cl + i;
          if (r < ep.M && cc < ep.M && (!diag_blk || cc >= r)) {
            const double h = ep.h_f64 ? ((const double*)ep.H)[(size_t)r * ep.ldh + cc]
                                      : (double)((const float*)ep.H)[(size_t)r * ep.ldh + cc];
            const float d = xs[i] + (cc == r ? thf : 0.f);
            pp[2] += (cc == r ? 1.f : 2.f) * d * (float)h;
          }
        }
      }
    }
    // rows 4 jh .. 4 jh + 15 of the block, mirrored
    __syncwarp();
    mirror_half(stage, Mp, orow0, ocol0, 4 * jh, diag_blk,
                [&](size_t off, float4 o) { store_out4<BF16>(ep, off, o); },
                [&](size_t off, float v) { store_out1<BF16>(ep, off, v); });
    __syncwarp();
  }
}

// GEMM2 epilogue of one warp for one 32 x 32 block, laid out as gemm1_pass
// (`yb`: s^2 (X Sigma) in the scratch tile): X_{n+1} = ca X + cb Sigma +
// cz Z (+ cj on the diagonal of the unpadded block).  Without products (mma
// false) the block is a copy of X and `yb` is not read.
template <bool BF16>
__device__ __forceinline__ void gemm2_pass(const Epi& ep, const float* __restrict__ yb, int ys,
                                           int orow0, int ocol0, bool diag_blk, bool mma,
                                           float ca, float cb, float cj, float cz,
                                           float* __restrict__ stage) {
  const int lane = threadIdx.x & 31;
  const int Mp = ep.Mp;
  const float is2 = ep.inv_s2;
  const int rs = lane >> 3, cl = 4 * (lane & 7);
  const size_t cbase = (size_t)ocol0 + cl;
  // four rows in flight per lane (three float4 operands each)
#pragma unroll
  for (int jh = 0; jh < 8; jh += 4) {
    float4 xx[4], ss[4], yy[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int rr = rs + 4 * (jh + j);
      const size_t off = (size_t)(orow0 + rr) * Mp + cbase;
      xx[j] = *reinterpret_cast<const float4*>(ep.X + off);
      if (mma) {
        ss[j] = *reinterpret_cast<const float4*>(ep.Sig + off);
        yy[j] = __ldcg(reinterpret_cast<const float4*>(yb + rr * ys + cl));
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = orow0 + rs + 4 * (jh + j);
      const size_t off = (size_t)r * Mp + cbase;
      float4 o = xx[j];
      if (mma) {
        o.x = fmaf(ca, xx[j].x, fmaf(cb, ss[j].x, cz * (yy[j].x * is2)));
        o.y = fmaf(ca, xx[j].y, fmaf(cb, ss[j].y, cz * (yy[j].y * is2)));
        o.z = fmaf(ca, xx[j].z, fmaf(cb, ss[j].z, cz * (yy[j].z * is2)));
        o.w = fmaf(ca, xx[j].w, fmaf(cb, ss[j].w, cz * (yy[j].w * is2)));
      }
      {
        float* st = stage + ((rs + 4 * (jh + j)) & 15) * kStageLd + cl;
        st[0] = o.x;
        st[1] = o.y;
        st[2] = o.z;
        st[3] = o.w;
      }
      if (!diag_blk) {
        store_out4<BF16>(ep, off, o);
      } else {
        const float ov[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int c = ocol0 + cl + i;
          if (c < r) continue;
          const float v = (mma && c == r && r < ep.M) ? ov[i] + cj : ov[i];
          store_out1<BF16>(ep, off + i, v);
        }
      }
    }
    // rows 4 jh .. 4 jh + 15 of the block, mirrored
    __syncwarp();
    mirror_half(stage, Mp, orow0, ocol0, 4 * jh, diag_blk,
                [&](size_t off, float4 o) { store_out4<BF16>(ep, off, o); },
                [&](size_t off, float v) { store_out1<BF16>(ep, off, v); });
    __syncwarp();
  }
}

// Plain-product epilogue (modes 5 and 6) of one warp for one 32 x 32 block:
// C = inv_s2 (A B) in FP32, laid out as gemm1_pass.  Mode 6 writes a block
// above the diagonal twice (direct and mirror, through `stage`).
template <bool MIRROR>
__device__ __forceinline__ void plain_pass(const Epi& ep, const float* __restrict__ yb, int ys,
                                           int orow0, int ocol0, bool diag_blk,
                                           float* __restrict__ stage) {
  const int lane = threadIdx.x & 31;
  const int rs = lane >> 3, cl = 4 * (lane & 7);
  const float sc = ep.inv_s2;
  // the whole block's loads in flight before its first store
  float4 yv[8];
#pragma unroll
  for (int j = 0; j < 8; ++j)
    yv[j] = __ldcg(reinterpret_cast<const float4*>(yb + (rs + 4 * j) * ys + cl));
#pragma unroll
  for (int jh = 0; jh < 8; jh += 4) {
    const float4* yy = yv + jh;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = orow0 + rs + 4 * (jh + j);
      const size_t off = (size_t)r * ep.Mp + ocol0 + cl;
      const float4 o = make_float4(yy[j].x * sc, yy[j].y * sc, yy[j].z * sc, yy[j].w * sc);
      if (MIRROR) {
        float* st = stage + (rs + 4 * j) * kStageLd + cl;
        st[0] = o.x;
        st[1] = o.y;
        st[2] = o.z;
        st[3] = o.w;
      }
      if (!diag_blk) {
        *reinterpret_cast<float4*>(ep.out + off) = o;
      } else {
        const float ov[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int c = ocol0 + cl + i;
          if (c < r) continue;
          ep.out[off + i] = ov[i];
        }
      }
    }
    if (MIRROR) {
      __syncwarp();
      mirror_half(stage, ep.Mp, orow0, ocol0, 4 * jh, diag_blk,
                  [&](size_t off, float4 o) { *reinterpret_cast<float4*>(ep.out + off) = o; },
                  [&](size_t off, float v) { ep.out[off] = v; });
      __syncwarp();
    }
  }
}

// Everything one tile needs: its block coordinates, operand maps, the
// epilogue pointers of its instance and the update coefficients.
struct TileCtx {
  int g;  // tile id (index of its partials)
  int I, J, nkb;
  bool skip;  // instance stopped: no work at all
  bool mma;   // products needed (false: identity copy of the iterate)
  const CUtensorMap *ah, *al, *bh, *bl;
  Epi ep;
  float ca, cb, cj, cz;
};

template <int MODE, bool BATCHED>
__device__ __forceinline__ void make_ctx(int t, const Epi& base, const CUtensorMap* mAh,
                                         const CUtensorMap* mAl, const CUtensorMap* mBh,
                                         const CUtensorMap* mBl, const BatchItem* items,
                                         const int* tile_inst, TileCtx& c) {
  c.ep = base;
  c.g = t;
  if (!BATCHED) {
    if (MODE == 5)
      tc_tile_full(t, base.Mp / BM, nj_blocks(base.Mp), c.I, c.J);
    else
      tc_tile(t, base.Mp / BM, nj_blocks(base.Mp), c.I, c.J);
    c.skip = false;
    c.ah = mAh;
    c.al = mAl;
    c.bh = mBh;
    c.bl = mBl;
  } else {
    if (base.order) c.g = t = base.order[t];
    const BatchItem& it = items[tile_inst[t]];
    State* st = it.st;
    c.skip = st->stopped != 0;
    const int par = st->parity;
    const CUtensorMap* maps = (const CUtensorMap*)it.maps;
    c.ep.st = st;
    c.ep.M = it.M;
    c.ep.Mp = it.Mp;
    c.ep.H = nullptr;
    if (MODE == 1) {
      // GEMM1 reads the current buffer and writes Sigma
      c.ep.X = it.X[par];
      c.ep.out = it.Sig;
      c.ep.out_h = it.Sh;
      c.ep.out_l = it.Sl;
      c.ah = c.bh = &maps[2 * par];
      c.al = c.bl = &maps[2 * par + 1];
    } else if (MODE == 2) {
      // the control kernel flipped the parity: read par^1, write par
      c.ep.X = it.X[par ^ 1];
      c.ep.Sig = it.Sig;
      c.ep.out = it.X[par];
      c.ep.out_h = it.Xh[par];
      c.ep.out_l = it.Xl[par];
      c.ah = &maps[2 * (par ^ 1)];
      c.al = &maps[2 * (par ^ 1) + 1];
      c.bh = &maps[4];
      c.bl = &maps[5];
    } else if (MODE == 4) {
      // stop-test product after a refinement step: A = D (halves at
      // kRefScale), B = s Delta, the third segment's B = kRefScale Delta
      // (slices 0 and 1); D1 = D64[par], the step's output
      const CUtensorMap* om = (const CUtensorMap*)it.oz_maps;
      c.ah = &om[kOzSlices];
      c.al = &om[kOzSlices + 1];
      c.bh = &om[kOzSlices + 2];
      c.bl = &om[kOzSlices + 3];
      c.ep.emaps = &om[kOzSlices + 4];
      c.ep.S64 = it.S64;
      c.ep.D64 = it.D64[par];
      c.ep.ld64 = it.M;
    } else {
      // refinement product (X = S - D) D: the iterate just evaluated is
      // par^1 (the control kernel flipped the parity), the step writes par
      const CUtensorMap* om = (const CUtensorMap*)it.oz_maps;
      c.ah = &om[kOzSlices + 2];
      c.al = &om[kOzSlices + 3];
      c.bh = &om[kOzSlices];
      c.bl = &om[kOzSlices + 1];
      c.ep.S64 = it.S64;
      c.ep.D64 = it.D64[par ^ 1];
      c.ep.Dn64 = it.D64[par];
      c.ep.rs_x = it.oz_xs;
      c.ep.rs_d = it.oz_rs;
      c.ep.ld64 = it.M;
    }
    tc_tile(t - it.tc_off, it.Mp / BM, nj_blocks(it.Mp), c.I, c.J);
  }
  const State* st = c.ep.st;
  c.mma = !c.skip && (MODE == 1 || MODE >= 5 || st->apply != 0);
  c.nkb = c.mma ? (MODE == 4 ? 3 : 1) * (c.ep.Mp / BK) : 0;
  c.ca = c.cb = c.cj = c.cz = 0.f;
  if (MODE == 2 && !c.skip) {
    const double th = st->theta, g3 = st->g3;
    c.ca = (float)(st->a + g3 * th * th);
    c.cb = (float)(st->b + g3 * th);
    c.cj = (float)st->xshift;
    c.cz = (float)g3;
  }
}

template <int MODE, bool BF16, bool BATCHED>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                   const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
                   const Epi ep, const BatchItem* items, const int* tile_inst) {
  if (!BATCHED && MODE < 5) {
    State* st = ep.st;
    if (st->stopped || st->timeout) return;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int KC = kc_stages<MODE>();

  // each stage has two halves, the hi operands and the lo operands, with a
  // full and an empty barrier each: the lo halves are needed only by the
  // cross products, so they are released (and refilled) ahead of the hi
  // halves, which the hi x hi pass at the end of the chunk still reads
  __shared__ __align__(8) uint64_t full_hi[kHiSlots], full_lo[kLoSlots];
  __shared__ __align__(8) uint64_t empty_hi[kHiSlots], empty_lo[kLoSlots];
  __shared__ __align__(8) uint64_t accf_bar[2];    // chunk in TMEM buffer b complete
  __shared__ __align__(8) uint64_t acce_bar[2];    // TMEM buffer b drained
  __shared__ __align__(8) uint64_t sfull_bar[2];   // scratch slot holds a finished tile
  __shared__ __align__(8) uint64_t sempty_bar[2];  // scratch slot consumed by the epilogue
  __shared__ __align__(8) uint64_t fin_bar;
  __shared__ __align__(8) uint64_t never_bar;      // no thread arrives on it (diagnostic)
  __shared__ uint32_t tmem_holder;
  __shared__ double red[2 * 4 * 5];
  __shared__ float epi_stage[4 * kStageFloats];  // one 16 x 32 staging buffer per epilogue warp
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kHiSlots; ++s) {
      mbar_init(&full_hi[s], 1);
      mbar_init(&empty_hi[s], 1);
    }
    for (int s = 0; s < kLoSlots; ++s) {
      mbar_init(&full_lo[s], 1);
      mbar_init(&empty_lo[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf_bar[b], 1);
      mbar_init(&acce_bar[b], 8);               // the eight drain warps
      mbar_init(&sfull_bar[b], 8);              // the eight drain warps
      mbar_init(&sempty_bar[b], kEpiThreads / 32);  // the four epilogue warps
    }
    mbar_init(&fin_bar, 1);
    mbar_init(&never_bar, 1);
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
  int* timeout_flag = BATCHED ? &items[0].st->timeout : &ep.st->timeout;
  const unsigned long long wlim = ep.wait_ns;

  if (warp < 4) {
    reg_dealloc<kCtlRegs>();
    if (warp == 0 && lane == 0) {
      // ---------------- TMA producer ----------------
      // Stage by stage, the lo part then the hi part (ring slots gs % kLoSlots
      // and gs % kHiSlots for global stage gs).
      uint32_t gs = 0;              // global stage counter
      uint32_t issued[2] = {0, 0};  // parts issued so far: lo, hi
      bool alive = true;
      for (int t = blockIdx.x; t < ep.ntiles && alive; t += gridDim.x) {
        TileCtx c;
        make_ctx<MODE, BATCHED>(t, ep, &mAh, &mAl, &mBh, &mBl, items, tile_inst, c);
        for (int kb = 0; kb < c.nkb && alive; ++kb, ++gs) {
          int kx = kb * BK;
          const CUtensorMap *ah = c.ah, *al = c.al, *bh = c.bh, *bl = c.bl;
          if (MODE == 4) {
            // K = [0, 3 Mp): A rows [D | Delta | Delta], B rows [Delta | D | Delta]
            // (maps: a* = D, b* = Delta, emaps = Delta at D's scale), so the
            // sum is D Delta + Delta D + Delta^2, all in the scale kRefScale s_Delta
            const int kseg = c.ep.Mp / BK, seg = kb / kseg;
            kx = (kb - seg * kseg) * BK;
            if (seg >= 1) {
              ah = c.bh;
              al = c.bl;
            }
            if (seg == 1) {
              bh = c.ah;
              bl = c.al;
            } else if (seg == 2) {
              bh = &c.ep.emaps[0];
              bl = &c.ep.emaps[1];
            }
          }
          for (int hi = 0; hi < 2; ++hi) {
            const int nsl = hi ? kHiSlots : kLoSlots;
            const uint32_t sl = gs % nsl, use = gs / nsl;
            uint64_t* emp = hi ? &empty_hi[sl] : &empty_lo[sl];
            uint64_t* ful = hi ? &full_hi[sl] : &full_lo[sl];
            if (use >= 1 && !mbar_wait(emp, (use - 1) & 1, wlim)) {
              atomicOr(timeout_flag, 1);
              alive = false;
              break;
            }
            const uint32_t dst = sbase + (hi ? sl : kHiSlots + sl) * kPartBytes;
            const CUtensorMap* am = hi ? ah : al;
            const CUtensorMap* bm = hi ? bh : bl;
            mbar_expect_tx(ful, kPartBytes);
            tma_load_2d(am, ful, dst, kx, c.I * BM);
            tma_load_2d(bm, ful, dst + kABytes, kx, c.J * BN);
            tma_load_2d(bm, ful, dst + kABytes + kBBytes / 2, kx, c.J * BN + 128);
            issued[hi] = gs + 1;
          }
          if (!alive) break;
        }
      }
      // every issued load must land before the CTA exits: the last uses of
      // each ring (earlier ones were waited on by the MMA warp before it
      // released their slots)
      for (int hi = 0; hi < 2; ++hi) {
        const uint32_t nsl = hi ? kHiSlots : kLoSlots;
        uint64_t* ful = hi ? full_hi : full_lo;
        const uint32_t n = issued[hi], first = n > nsl ? n - nsl : 0;
        for (uint32_t k = first; k < n; ++k)
          if (!mbar_wait(&ful[k % nsl], (k / nsl) & 1, wlim)) atomicOr(timeout_flag, 1);
      }
    } else if (warp == 1 && lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t idesc = idesc_f16(BF16 ? 1 : 0);
      uint32_t g = 0, qc = 0;  // global stage and chunk counters
      bool alive = true;
      for (int t = blockIdx.x; t < ep.ntiles && alive; t += gridDim.x) {
        TileCtx c;
        make_ctx<MODE, BATCHED>(t, ep, &mAh, &mAl, &mBh, &mBl, items, tile_inst, c);
        const int nchunk = c.nkb / KC;
        for (int ch = 0; ch < nchunk && alive; ++ch, ++qc) {
          const uint32_t b = qc & 1;
          if (qc >= 2 && !mbar_wait(&acce_bar[b], ((qc >> 1) - 1) & 1, wlim)) {
            atomicOr(timeout_flag, 1);
            alive = false;
            break;
          }
          tc_fence_after();
          const uint32_t acc = tmem + b * 256;
          // the cross products of the chunk first (they round at their own
          // scale), releasing each stage's lo part; then hi x hi, releasing
          // the hi parts
          for (int ks = 0; ks < KC; ++ks) {
            const uint32_t gs = g + ks, sl = gs % kLoSlots, sh = gs % kHiSlots;
            if (!mbar_wait(&full_lo[sl], (gs / kLoSlots) & 1, wlim) ||
                !mbar_wait(&full_hi[sh], (gs / kHiSlots) & 1, wlim)) {
              atomicOr(timeout_flag, 1);
              alive = false;
              break;
            }
            tc_fence_after();
            const uint32_t a_h = sbase + sh * kPartBytes, b_h = a_h + kABytes;
            const uint32_t a_l = sbase + (kHiSlots + sl) * kPartBytes, b_l = a_l + kABytes;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint32_t off = kk * 32;  // 16 halves = 32 B inside the 64 B swizzle row
              umma(acc, sdesc(a_h + off), sdesc(b_l + off), idesc, (ks == 0 && kk == 0) ? 0u : 1u);
              umma(acc, sdesc(a_l + off), sdesc(b_h + off), idesc, 1u);
            }
            umma_commit(&empty_lo[sl]);
          }
          if (!alive) break;
          for (int ks = 0; ks < KC; ++ks) {
            const uint32_t sh = (g + ks) % kHiSlots;
            const uint32_t a_h = sbase + sh * kPartBytes, b_h = a_h + kABytes;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint32_t off = kk * 32;
              umma(acc, sdesc(a_h + off), sdesc(b_h + off), idesc, 1u);
            }
            umma_commit(&empty_hi[sh]);
          }
          g += KC;
          umma_commit(&accf_bar[b]);
        }
      }
      // every MMA issued here must be complete before TMEM is freed
      umma_commit(&fin_bar);
      if (!mbar_wait(&fin_bar, 0, wlim)) atomicOr(timeout_flag, 1);
    }
  } else if (warp < kEpiWarp0) {
    reg_alloc<drain_regs<BATCHED>()>();
    // ---------------- drain (warps 4..11) ----------------
    // TMEM lane quarter is fixed by the warp's rank within its warpgroup
    const int dw = warp - 4, q = warp & 3, half = dw >> 2;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    float* slots = ep.scratch + (size_t)blockIdx.x * 2 * kSlotFloats;
    uint32_t qc = 0, u = 0;
    bool alive = true;
    if (ep.stall) {
      // diagnostic: a wait that no thread will satisfy, to exercise the
      // bounded-wait path of every role (see gcp_debug_timeout)
      if (!__all_sync(0xffffffffu, mbar_wait(&never_bar, 0, wlim))) {
        if (lane == 0) atomicOr(timeout_flag, 1);
        alive = false;
      }
    }
    for (int t = blockIdx.x; t < ep.ntiles && alive; t += gridDim.x) {
      TileCtx c;
      make_ctx<MODE, BATCHED>(t, ep, &mAh, &mAl, &mBh, &mBl, items, tile_inst, c);
      if (c.skip || c.nkb == 0) continue;  // no products: nothing to hand over
      float acc[128];
#pragma unroll
      for (int k = 0; k < 128; ++k) acc[k] = 0.f;
      const int nchunk = c.nkb / KC;
      for (int ch = 0; ch < nchunk; ++ch, ++qc) {
        const uint32_t b = qc & 1;
        // warp-uniform: tcgen05.ld below is a warp-collective instruction
        if (!__all_sync(0xffffffffu, mbar_wait(&accf_bar[b], (qc >> 1) & 1, wlim))) {
          if (lane == 0) atomicOr(timeout_flag, 1);
          alive = false;
          break;
        }
        tc_fence_after();
        const uint32_t base = tmem + lane_base + b * 256 + half * 128;
#pragma unroll
        for (int part = 0; part < 4; ++part) {
          uint32_t r[32];
          tmem_ld32(base + part * 32, r);
          tmem_ld_wait();
#pragma unroll
          for (int k = 0; k < 32; ++k) acc[part * 32 + k] += __uint_as_float(r[k]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce_bar[b]);
      }
      if (!alive) break;
      if constexpr (MODE == 5) {
        // a non-symmetric plain product's epilogue is a scaled copy: the
        // drain stores its row's 128 columns itself (the same products as
        // the epilogue's, C = inv_s2 (A B)), skipping the scratch round trip
        const int col0 = c.J * BN + half * 128;
        if (col0 < c.ep.Mp) {
          const float sc = c.ep.inv_s2;
          float4* dst = reinterpret_cast<float4*>(
              c.ep.out + (size_t)(c.I * BM + 32 * q + lane) * c.ep.Mp + col0);
#pragma unroll
          for (int k = 0; k < 32; ++k)
            dst[k] = make_float4(acc[4 * k] * sc, acc[4 * k + 1] * sc, acc[4 * k + 2] * sc,
                                 acc[4 * k + 3] * sc);
        }
        continue;
      }
      // hand the tile to the epilogue warps through scratch slot u & 1
      const uint32_t slot = u & 1;
      if (u >= 2 && !__all_sync(0xffffffffu, mbar_wait(&sempty_bar[slot], ((u >> 1) - 1) & 1, wlim))) {
        if (lane == 0) atomicOr(timeout_flag, 1);
        alive = false;
        break;
      }
      // row-major: a thread's 128 columns of its row
      float* tile = slots + slot * kSlotFloats;
      float4* dst = reinterpret_cast<float4*>(tile + (size_t)(32 * q + lane) * BN + half * 128);
#pragma unroll
      for (int k = 0; k < 32; ++k)
        __stcg(dst + k, make_float4(acc[4 * k], acc[4 * k + 1], acc[4 * k + 2], acc[4 * k + 3]));
      __threadfence_block();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sfull_bar[slot]);
      ++u;
    }
  } else {
    if constexpr (epi_regs<BATCHED>() > 128)
      reg_alloc<epi_regs<BATCHED>()>();
    else
      reg_dealloc<epi_regs<BATCHED>()>();
    // ---------------- epilogue (warps 12..15) ----------------
    // (none in mode 5: the drain warps store the product)
    const int e = warp - kEpiWarp0;  // every fourth block of a tile; prefetches rows 32 e..
    const float* slots = ep.scratch + (size_t)blockIdx.x * 2 * kSlotFloats;
    uint32_t u = 0, nred = 0;
    // Batched (short-K) tiles, whose epilogue bounds the launch: L2
    // prefetch of the FP32 rows this warp reads from HBM in GEMM1 and GEMM2
    // (X, and Sigma when GEMM2 has products): row 32 e + lane of a tile,
    // from the first 128-column block on or above the diagonal to the
    // tile's last column, one bulk prefetch per operand, issued for the
    // next tile halfway through the current one.
    auto prefetch_rows = [&](const TileCtx& q) {
      if constexpr (MODE == 1 || MODE == 2) {
        if (q.skip) return;
        const int h0 = 2 * q.J >= q.I ? 0 : 1;
        const int cs = q.J * BN + 128 * h0, ce = q.J * BN + BN < q.ep.Mp ? q.J * BN + BN : q.ep.Mp;
        if (ce <= cs) return;
        const size_t off = (size_t)(q.I * BM + 32 * e + lane) * q.ep.Mp + cs;
        const uint32_t bytes = (uint32_t)(ce - cs) * sizeof(float);
        l2_prefetch(q.ep.X + off, bytes);
        if (MODE == 2 && q.mma) l2_prefetch(q.ep.Sig + off, bytes);
      }
    };
    int pf_t = -1;  // the tile whose rows were prefetched ahead
    for (int t = blockIdx.x; MODE != 5 && t < ep.ntiles; t += gridDim.x) {
      TileCtx c;
      make_ctx<MODE, BATCHED>(t, ep, &mAh, &mAl, &mBh, &mBl, items, tile_inst, c);
      if (c.skip) continue;  // uniform over the CTA
      if (BATCHED && t != pf_t) prefetch_rows(c);
      const bool has = c.nkb > 0;
      const uint32_t slot = u & 1;
      bool ok = !(*(volatile int*)timeout_flag);
      if (has && ok) {
        ok = __all_sync(0xffffffffu, mbar_wait(&sfull_bar[slot], (u >> 1) & 1, wlim));
        if (!ok && lane == 0) atomicOr(timeout_flag, 1);
      }
      const float* tile = slots + slot * kSlotFloats;
      double dpart[2] = {0.0, 0.0};  // diagonal sums (FP64)
      float pp[3] = {0.f, 0.f, 0.f};  // element sums (FP32 per lane)
      // does the tile reach the diagonal? (uniform: decides the FP64 sums)
      const bool tile_diag = (2 * c.J == c.I) || (2 * c.J + 1 == c.I);
      if (ok) {
        float thf = 0.f, f2th = 0.f, thtb = 0.f;
        if constexpr (MODE == 1) {
          const double th = c.ep.st->theta;
          thf = (float)th;
          f2th = (float)(2.0 * th);
          thtb = (float)(th * (1.0 - th));
        }
        // The tile's 32 x 32 blocks that the product writes (stripe s =
        // rows 32 s.., column block p), taken in stripe order and dealt
        // round-robin to the four epilogue warps: on a tile that reaches the
        // diagonal the stripes hold different numbers of blocks, and one
        // warp per stripe would leave the others waiting at the tile's
        // barrier.
        int q = 0;
#pragma unroll 1
        for (int k = 0; k < 32; ++k) {
          if ((MODE == 1 || MODE == 2) && BATCHED && k == 16 && t + (int)gridDim.x < ep.ntiles) {
            TileCtx cn;
            make_ctx<MODE, BATCHED>(t + gridDim.x, ep, &mAh, &mAl, &mBh, &mBl, items, tile_inst,
                                    cn);
            prefetch_rows(cn);
            pf_t = t + gridDim.x;
          }
          const int sp = k >> 3, p = k & 7;
          const int half = p >> 2, part = p & 3;
          const int jb = 2 * c.J + half;  // 128-column block
          // below the diagonal: the mirror of another tile (all tiles are
          // computed in mode 5, a non-symmetric product)
          if (MODE != 5 && jb < c.I) continue;
          if (MODE != 5 && jb == c.I && part < sp) continue;
          if (128 * jb >= c.ep.Mp) continue;  // past the matrix (last column block)
          if ((q++ & 3) != e) continue;
          const bool dblk = MODE != 5 && jb == c.I && part == sp;
          const int row0 = c.I * BM + 32 * sp;
          const int cl0 = half * 128 + part * 32;  // tile-local column of the block
          const int c0 = c.J * BN + cl0;
          // rows row0.., columns c0.. of the row-major scratch tile (and
          // their mirror, through this warp's staging buffer)
          const float* yd = tile + (size_t)(32 * sp) * BN + cl0;
          float* stage = epi_stage + e * kStageFloats;
          if constexpr (MODE == 1) {
            gemm1_pass<BF16>(c.ep, yd, BN, row0, c0, dblk, thf, f2th, thtb, pp, dpart, stage);
          } else if constexpr (MODE == 2) {
            gemm2_pass<BF16>(c.ep, yd, BN, row0, c0, dblk, c.mma, c.ca, c.cb, c.cj, c.cz, stage);
          } else if constexpr (MODE == 5) {
            plain_pass<false>(c.ep, yd, BN, row0, c0, false, stage);
          } else if constexpr (MODE == 6) {
            plain_pass<true>(c.ep, yd, BN, row0, c0, dblk, stage);
          } else if constexpr (MODE == 4) {
            const float inv = (float)(1.0 / (kRefScale * check_delta_scale(c.ep.st->R)));
            check_seg(c.ep, row0 + lane, c0, jb == c.I, yd + lane * BN, inv, pp, dpart);
          } else {
            refine_seg(c.ep, row0 + lane, c0, jb == c.I, yd + lane * BN);
          }
        }
      }
      if (has) {
        __syncwarp();
        if (lane == 0 && ok) mbar_arrive(&sempty_bar[slot]);
        ++u;
      }
      if (MODE == 1 || MODE == 4) {
        // per-tile partials: element sums in FP32 (a float shuffle tree),
        // the diagonal sums in FP64 only on tiles that reach the diagonal
        // (FP64 arithmetic is slow on this part); lanes of warp 12 add the
        // four warps' rows in a fixed order.  The table is double-buffered
        // by the count of reduced tiles, so one barrier per tile suffices.
        const float s2 = warp_sum_f(pp[0]), s3 = warp_sum_f(pp[1]), s4 = warp_sum_f(pp[2]);
        double d0 = 0.0, d1 = 0.0;
        if (tile_diag) {
          d0 = warp_sum(dpart[0]);
          d1 = warp_sum(dpart[1]);
        }
        double* r = red + (nred & 1) * 20;
        if (lane == 0) {
          r[e * 5] = d0;
          r[e * 5 + 1] = d1;
          r[e * 5 + 2] = (double)s2;
          r[e * 5 + 3] = (double)s3;
          r[e * 5 + 4] = (double)s4;
        }
      }
      // one barrier per tile: publishes the table and decides, uniformly,
      // whether the epilogue warps go on
      const bool stop = bar_red_or(kEpiBarrier, kEpiThreads, !ok);
      if ((MODE == 1 || MODE == 4) && e == 0 && lane < kPartFields) {
        const double* r = red + (nred & 1) * 20;
        double sacc = 0.0;
        if (lane < 5)
          for (int w = 0; w < 4; ++w) sacc += r[w * 5 + lane];
        ep.part[(size_t)c.g * kPartFields + lane] = sacc;
      }
      ++nred;
      if (stop) break;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols));
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode(char* err, int errlen) {
  static EncodeTiledFn fn = nullptr;
  if (fn) return fn;
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                   cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
    snprintf(err, errlen, "cuTensorMapEncodeTiled unavailable (%s)", cudaGetErrorString(e));
    return nullptr;
  }
  fn = (EncodeTiledFn)p;
  return fn;
}

// box_k = 32 (64-byte rows, SWIZZLE_64B) or 64 (128-byte rows, SWIZZLE_128B).
int encode_map(CUtensorMap* m, const void* ptr, int Mp, int bf16, char* err, int errlen,
               int box_k = BK) {
  EncodeTiledFn enc = get_encode(err, errlen);
  if (!enc) return 1;
  if (((uintptr_t)ptr & 15u) != 0 || ((size_t)Mp * 2) % 16 != 0 || Mp % BM != 0) {
    snprintf(err, errlen, "tensor map: misaligned operand or size");
    return 1;
  }
  cuuint64_t dims[2] = {(cuuint64_t)Mp, (cuuint64_t)Mp};
  cuuint64_t strides[1] = {(cuuint64_t)Mp * 2};
  if (box_k != 32 && box_k != 64) {
    snprintf(err, errlen, "tensor map: unsupported box width");
    return 1;
  }
  cuuint32_t box[2] = {(cuuint32_t)box_k, (cuuint32_t)BM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                   const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   box_k == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    snprintf(err, errlen, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return 1;
  }
  return 0;
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

// Launch on at most one CTA per SM (persistent tiles).  `ep.scratch` must
// hold tc_scratch_bytes(): two tile slots for every CTA of the grid.
template <int MODE, bool BF16, bool BATCHED>
int launch_tc(const TcOperands* A, const TcOperands* B, Epi ep, const BatchItem* items,
              const int* tile_inst, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<MODE, BF16, BATCHED>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return 1;
    // the register split must fit the pool the CTA is launched with, or
    // the drain warpgroups' setmaxnreg.inc would wait forever
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, tc_gemm_kernel<MODE, BF16, BATCHED>) != cudaSuccess ||
        fa.numRegs * kThreads < (int)split_regs<BATCHED>())
      return 1;
    attr = true;
  }
  if (!ep.scratch) return 1;
  if (ep.wait_ns == 0) ep.wait_ns = kWaitNs;
  const int grid = ep.ntiles < sm_count() ? ep.ntiles : sm_count();
  if (grid <= 0) return 0;
  if (BATCHED) {
    CUtensorMap dummy;
    memset(&dummy, 0, sizeof dummy);
    tc_gemm_kernel<MODE, BF16, true><<<grid, kThreads, kSmemBytes, s>>>(dummy, dummy, dummy, dummy,
                                                                     ep, items, tile_inst);
  } else {
    tc_gemm_kernel<MODE, BF16, false><<<grid, kThreads, kSmemBytes, s>>>(A->hi, A->lo, B->hi, B->lo,
                                                                      ep, nullptr, nullptr);
  }
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 1;
}
}  // namespace

int tc_pad(int M) { return ((M + BM - 1) / BM) * BM; }

size_t tc_scratch_bytes() { return (size_t)sm_count() * 2 * kSlotFloats * sizeof(float); }

int tc_encode_map(void* map, const void* ptr, int Mp, int bf16, char* err, int errlen, int box_k) {
  return encode_map((CUtensorMap*)map, ptr, Mp, bf16, err, errlen, box_k);
}

int tc_num_tiles(int Mp) {
  const int NI = Mp / BM, NJ = nj_blocks(Mp);
  int n = 0;
  for (int j = 0; j < NJ; ++j) n += (2 * j + 2 < NI ? 2 * j + 2 : NI);
  return n;
}

int tc_make_operands(TcOperands** op, const void* hi, const void* lo, int Mp, int bf16, char* err,
                     int errlen) {
  TcOperands* o = new TcOperands;
  if (encode_map(&o->hi, hi, Mp, bf16, err, errlen) || encode_map(&o->lo, lo, Mp, bf16, err, errlen)) {
    delete o;
    return 1;
  }
  *op = o;
  return 0;
}

void tc_free_operands(TcOperands* op) { delete op; }

int tc_launch_gemm1(const TcOperands* opX, const float* X, float* Sig, void* Sh, void* Sl, int M,
                    int Mp, const void* H, int h_f64, int ldh, double* part, State* st, int bf16,
                    float split_scale, float* scratch, cudaStream_t s, unsigned long long wait_ns,
                    int stall) {
  Epi ep{};
  ep.scratch = scratch;
  ep.wait_ns = wait_ns;
  ep.stall = stall;
  ep.X = X;
  ep.Sig = nullptr;
  ep.out = Sig;
  ep.out_h = Sh;
  ep.out_l = Sl;
  ep.H = H;
  ep.h_f64 = h_f64;
  ep.ldh = ldh;
  ep.part = part;
  ep.st = st;
  ep.M = M;
  ep.Mp = Mp;
  ep.ntiles = tc_num_tiles(Mp);
  ep.split_scale = split_scale;
  ep.inv_s2 = 1.0f / (split_scale * split_scale);
  return bf16 ? launch_tc<1, true, false>(opX, opX, ep, nullptr, nullptr, s)
              : launch_tc<1, false, false>(opX, opX, ep, nullptr, nullptr, s);
}

int tc_launch_gemm2(const TcOperands* opS, const TcOperands* opX, const float* X, const float* Sig,
                    float* Xn, void* Xnh, void* Xnl, int M, int Mp, State* st, int bf16,
                    float split_scale, float* scratch, cudaStream_t s) {
  Epi ep{};
  ep.scratch = scratch;
  ep.X = X;
  ep.Sig = Sig;
  ep.out = Xn;
  ep.out_h = Xnh;
  ep.out_l = Xnl;
  ep.H = nullptr;
  ep.part = nullptr;
  ep.st = st;
  ep.M = M;
  ep.Mp = Mp;
  ep.ntiles = tc_num_tiles(Mp);
  ep.split_scale = split_scale;
  ep.inv_s2 = 1.0f / (split_scale * split_scale);
  return bf16 ? launch_tc<2, true, false>(opX, opS, ep, nullptr, nullptr, s)
              : launch_tc<2, false, false>(opX, opS, ep, nullptr, nullptr, s);
}

void tc_set_smem_attrs() {}

int tc_launch_mcweeny64(const TcOperands* opX, const TcOperands* opD, const double* S64,
                        const double* D64, double* Dn64, const double* xscale,
                        const double* dscale, int M, int Mp, State* st, float* scratch,
                        cudaStream_t s) {
  Epi ep{};
  ep.scratch = scratch;
  ep.st = st;
  ep.M = M;
  ep.Mp = Mp;
  ep.ntiles = tc_num_tiles(Mp);
  ep.split_scale = 1.0f;
  ep.inv_s2 = 1.0f;
  ep.S64 = S64;
  ep.D64 = D64;
  ep.Dn64 = Dn64;
  ep.rs_x = xscale;
  ep.rs_d = dscale;
  ep.ld64 = M;
  return launch_tc<3, false, false>(opX, opD, ep, nullptr, nullptr, s);
}

int tc_make_device_maps(void** dev, const void* hi, const void* lo, int Mp, char* err,
                        int errlen) {
  CUtensorMap m[2];
  if (encode_map(&m[0], hi, Mp, 0, err, errlen) || encode_map(&m[1], lo, Mp, 0, err, errlen))
    return 1;
  if (cudaMalloc(dev, sizeof m) != cudaSuccess ||
      cudaMemcpy(*dev, m, sizeof m, cudaMemcpyHostToDevice) != cudaSuccess) {
    snprintf(err, errlen, "device tensor maps: %s", cudaGetErrorString(cudaGetLastError()));
    return 1;
  }
  return 0;
}

int tc_launch_check(const TcOperands* opD, const TcOperands* opDelta, const void* emaps,
                    const double* S64, const double* D1, double* part, int M, int Mp, State* st,
                    float* scratch, cudaStream_t s) {
  Epi ep{};
  ep.scratch = scratch;
  ep.emaps = (const CUtensorMap*)emaps;
  ep.st = st;
  ep.M = M;
  ep.Mp = Mp;
  ep.ntiles = tc_num_tiles(Mp);
  ep.split_scale = 1.0f;
  ep.inv_s2 = 1.0f;
  ep.part = part;
  ep.S64 = S64;
  ep.D64 = D1;
  ep.ld64 = M;
  return launch_tc<4, false, false>(opD, opDelta, ep, nullptr, nullptr, s);
}

int tc_launch_product(const TcOperands* A, const TcOperands* B, float* C, int Mp, int symmetric,
                      float inv_scale, State* st, float* scratch, cudaStream_t s) {
  Epi ep{};
  ep.scratch = scratch;
  ep.st = st;
  ep.M = Mp;
  ep.Mp = Mp;
  ep.out = C;
  ep.split_scale = 1.0f;
  ep.inv_s2 = inv_scale;
  if (symmetric) {
    ep.ntiles = tc_num_tiles(Mp);
    return launch_tc<6, false, false>(A, B, ep, nullptr, nullptr, s);
  }
  ep.ntiles = (Mp / BM) * nj_blocks(Mp);
  return launch_tc<5, false, false>(A, B, ep, nullptr, nullptr, s);
}

size_t tc_map_bytes() { return 6 * sizeof(CUtensorMap); }

// Host images of the six tensor maps of one batched instance.
int tc_build_batch_maps(void* maps_host, const BatchItem& it, int bf16, char* err, int errlen) {
  CUtensorMap* m = (CUtensorMap*)maps_host;
  const void* ptrs[6] = {it.Xh[0], it.Xl[0], it.Xh[1], it.Xl[1], it.Sh, it.Sl};
  for (int k = 0; k < 6; ++k)
    if (encode_map(&m[k], ptrs[k], it.Mp, bf16, err, errlen)) return 1;
  return 0;
}

int tc_tile_cost(int Mp, int local) {
  int I, J;
  tc_tile(local, Mp / BM, nj_blocks(Mp), I, J);
  int c = Mp / 128;
  for (int sp = 0; sp < 4; ++sp)
    for (int p = 0; p < 8; ++p) {
      const int jb = 2 * J + (p >> 2), part = p & 3;
      if (jb < I || (jb == I && part < sp) || 128 * jb >= Mp) continue;
      c += (jb == I && part == sp) ? 1 : 2;
    }
  return c;
}

int tc_launch_batch_gemm(int mode, const BatchItem* items, int batch, const int* tile_inst,
                         const int* order, int ntiles, double* part, int bf16, float split_scale,
                         float* scratch, cudaStream_t s) {
  (void)batch;
  Epi ep{};
  ep.scratch = scratch;
  ep.order = order;
  ep.part = part;
  ep.ntiles = ntiles;
  ep.split_scale = split_scale;
  ep.inv_s2 = 1.0f / (split_scale * split_scale);
  if (mode == 1)
    return bf16 ? launch_tc<1, true, true>(nullptr, nullptr, ep, items, tile_inst, s)
                : launch_tc<1, false, true>(nullptr, nullptr, ep, items, tile_inst, s);
  if (mode == 3 || mode == 4) {
    // refinement and stop-test products: fp16 halves, scales carried by the
    // operands
    ep.split_scale = 1.0f;
    ep.inv_s2 = 1.0f;
    return mode == 3 ? launch_tc<3, false, true>(nullptr, nullptr, ep, items, tile_inst, s)
                     : launch_tc<4, false, true>(nullptr, nullptr, ep, items, tile_inst, s);
  }
  return bf16 ? launch_tc<2, true, true>(nullptr, nullptr, ep, items, tile_inst, s)
              : launch_tc<2, false, true>(nullptr, nullptr, ep, items, tile_inst, s);
}

}  // namespace gcp
