// Split-precision tensor-core products of one GCP step (sm_103a: tcgen05 +
// TMEM + TMA), with the step's elementwise work fused into the epilogues:
// mode 1 GEMM1, mode 2 GEMM2 of the split phase; mode 3 the product of an
// exact-slice refinement step, mode 4 the stop-test product after it
// (W = D1^2 - D^2 over a K = 3M concatenation of operands).
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
// Accumulation.  The tensor cores add into their FP32 accumulator with
// truncation; over a long K that biases every sum toward zero (measured
// ~6e-5 relative at K = 8192 for same-sign sums).  So the accumulator only
// ever holds one K chunk of 128 (24 MMAs; 32 in the refinement product):
// eight drain warps move each chunk from TMEM into FP32 registers with
// round-to-nearest adds while the MMA warp fills the other of two TMEM
// buffers.  (Chunks of 64 cost 16% more time in GEMM1 at M = 8192 for no
// measurable gain in accuracy; longer first chunks of a tile, which would
// keep the MMAs going through more of the previous tile's epilogue, moved
// the subspace error past 1e-6 at M = 8192.)
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
// upper block triangle.  Three warpgroups: in the first, warp 0 lane 0
// issues TMA loads (SWIZZLE_64B, 32-wide K blocks, a 4-stage ring of 48 KB
// stages) and warp 1 lane 0 issues tcgen05.mma (warps 2-3 idle); warps
// 4-11 drain TMEM and run the epilogue (warp w reads TMEM lanes 32(w%4)..
// and columns 128((w-4)/4)..).  The first warpgroup hands registers to the
// other two (setmaxnreg: 40 and 232 a thread against 168 at launch), which
// hold the 128 x 256 FP32 accumulator, 128 values a thread, without
// spilling.  Blocks below the diagonal inside a tile are skipped in the
// epilogue; every element above the diagonal is stored twice (direct and
// mirrored).  Every wait is bounded
// (2 s); on expiry the kernel records State::timeout and winds down, still
// freeing its TMEM.
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
constexpr int BM = 128, BN = 256, BK = 32, STAGES = 4;
// K chunk per TMEM drain = kc_stages * BK: 128 for the split phase; 32 for
// the FP64 refinement product (mode 3), whose trace must hold to ~1e-10:
// the truncation inside a chunk biases the diagonal of (S - D) D toward
// zero by about (MMAs per chunk) 2^-25, and 24 MMAs per chunk moved
// Tr D_{n+1} by ~1e-9 at M = 8192.
template <int MODE>
__host__ __device__ constexpr int kc_stages() {
  return MODE == 3 ? 1 : 4;
}
constexpr int kThreads = 384;
constexpr uint32_t kCtlRegs = 40, kDrainRegs = 232;  // per thread, after setmaxnreg
static_assert(128 * kCtlRegs + 256 * kDrainRegs <= 65536, "register split");
constexpr uint32_t kABytes = BM * BK * 2;                     // 8 KB
constexpr uint32_t kBBytes = BN * BK * 2;                     // 16 KB
constexpr uint32_t kStageBytes = 2 * kABytes + 2 * kBBytes;  // 48 KB
constexpr uint32_t kTpBytes = 8 * 32 * 32 * 4;  // one 32 x 32 float block per drain warp
// The split GEMMs' epilogues use the transposition buffers; the refinement
// product keeps that shared memory as L1 cache for its row-wise FP64 loads.
template <int MODE>
__host__ __device__ constexpr uint32_t smem_bytes() {
  return STAGES * kStageBytes + (MODE == 1 || MODE == 2 ? kTpBytes : 0u) + 1024;
}
static_assert(smem_bytes<1>() + 768 <= 227 * 1024, "shared memory per CTA");
constexpr uint32_t kTmemCols = 512;  // two 256-column accumulator buffers

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
};

// Linear tile index -> (I, J): I a 128-row block, J a 256-column block,
// kept when the tile reaches the upper block triangle (I < 2J + 2, i.e.
// J >= floor(I / 2)).  Order: super-columns of kGroupJ column blocks; in
// each, row block by row block, the super-column's tiles of that row.  The
// CTAs working at the same time then share a few A panels (rows) and the
// super-column's B panels, which stay in L2 while the CTAs stream along K.
constexpr int kGroupJ = 8;
__device__ __forceinline__ void tc_tile(int t, int NI, int NJ, int& I, int& J) {
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

// Refinement-product epilogue of one thread: its row, 128 columns of one
// 128-block (jb = 2J + half), values acc[] = (A B)_row,c in the slice scale.
// McWeeny refinement step in FP64 (Eq. mcweeny3): with S = D^2 exact and
// X = S - D small, 3D^2 - 2D^3 = S - 2 X D; the product Z = X D only needs
// the relative accuracy of the split product because |X| is small.  The
// general step of Eq. hpcp3 is the same plus (1 - 2c)(D - S); the control
// kernel sets c within 1/2 +- 0.05 to put Tr D+ back at N.
__device__ __forceinline__ void refine_row(const Epi& ep, int row, int c_base, bool diag_blk,
                                           const float (&acc)[128]) {
  if (row >= ep.M) return;
  const double wr = 1.0 / (kRefScale * ep.rs_x[row]);  // powers of two: exact
  const double g = ep.st->a;
#pragma unroll
  for (int k = 0; k < 128; ++k) {
    const int c = c_base + k;
    if (c >= ep.M || (diag_blk && c < row)) continue;
    const size_t o = (size_t)row * ep.ld64 + c;
    const double sv = ep.S64[o];
    const double v = sv - 2.0 * (wr * ep.rs_d[c]) * (double)acc[k] - g * (sv - ep.D64[o]);
    ep.Dn64[o] = v;
    if (c != row) ep.Dn64[(size_t)c * ep.ld64 + row] = v;
  }
}

// Stop-test epilogue of one thread after a refinement step D -> D1 (mode 4):
// acc[] = kRefScale s_Delta W_row,c with W = D1^2 - D^2 = D Delta + Delta D +
// Delta^2, Delta = D1 - D; with S = D^2 exact, D1^2 - D1 = S + W - D1 is
// formed in FP64 (S and D1 are O(1), the result is ~R1).  Sums: the
// residual R1^2 (FP32 per lane, weight 2 above the diagonal), Tr D1 and
// Tr D1^2 = Tr S + Tr W (FP64, diagonal only).
__device__ __forceinline__ void check_row(const Epi& ep, int row, int c_base, bool diag_blk,
                                          const float (&acc)[128], float inv_scale,
                                          float (&pp)[3], double (&dpart)[5]) {
  if (row >= ep.M) return;
  // fully unrolled: acc[] stays in registers
#pragma unroll
  for (int k = 0; k < 128; ++k) {
    const int c = c_base + k;
    if (c >= ep.M || (diag_blk && c < row)) continue;
    const size_t o = (size_t)row * ep.ld64 + c;
    const double sw = ep.S64[o] + (double)(acc[k] * inv_scale);  // D1^2, exact scaling
    const double d1 = ep.D64[o];
    const float x1 = (float)(sw - d1);
    pp[1] = fmaf((c == row ? 1.f : 2.f) * x1, x1, pp[1]);
    if (c == row) {
      dpart[0] += d1;
      dpart[1] += sw;
    }
  }
}

// GEMM1 epilogue of one warp for one 32 x 32 block: rows row0..row0+31,
// columns c0..c0+31; the caller has written s^2 (X X)_{row0+lane, c0+k} to
// row `lane` of the warp's shared buffer `tp` (lane = row, as the
// accumulator comes out of TMEM; 4-float groups XOR-swizzled by row), and
// the block is read back with eight lanes per row and four consecutive
// columns per lane, so that the X loads and the direct stores of Sigma and
// its halves are whole 128-byte row segments; Sigma goes back to `tp` and
// the mirrored stores read it with eight lanes per column.
// Blocks on the diagonal take an element-wise path (upper triangle only).
// The XOR key (r ^ r >> 2) & 7 takes eight distinct values over any eight
// consecutive rows (float4 rows written by lanes = rows) and over rows
// 4g + i, g = 0..7 (the mirrored reads): both are conflict-free.
__device__ __forceinline__ int tp_idx(int r, int c) {
  return r * 32 + ((((c >> 2) ^ ((r ^ (r >> 2)) & 7)) << 2) | (c & 3));
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

template <bool BF16>
__device__ __forceinline__ void gemm1_block(const Epi& ep, int row0, int c0, bool diag_blk,
                                            float thf, float f2th, float thtb, float (&pp)[3],
                                            double (&dpart)[5], float* tp) {
  const int lane = threadIdx.x & 31;
  const int Mp = ep.Mp;
  const float is2 = ep.inv_s2;
  __syncwarp();
  if (!diag_blk) {
    // every element lies above the diagonal (weight 2, mirrored)
    const int rs = lane >> 3, cl = 4 * (lane & 7);
    const size_t cbase = (size_t)c0 + cl;
    // all eight X loads in flight before the first store (loads issued
    // after stores queue behind them)
    float4 xx[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      xx[j] = *reinterpret_cast<const float4*>(ep.X + (size_t)(row0 + rs + 4 * j) * Mp + cbase);
#pragma unroll
    for (int jh = 0; jh < 8; jh += 4) {
      const float4* x = xx + jh;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int rr = rs + 4 * (jh + j);
        const size_t off = (size_t)(row0 + rr) * Mp + cbase;
        const float4 a = *reinterpret_cast<const float4*>(&tp[tp_idx(rr, cl)]);
        float4 o;
        o.x = fmaf(f2th, x[j].x, a.x * is2);  // Sigma = 2 theta X + Y
        o.y = fmaf(f2th, x[j].y, a.y * is2);
        o.z = fmaf(f2th, x[j].z, a.z * is2);
        o.w = fmaf(f2th, x[j].w, a.w * is2);
        const float ex = o.x - x[j].x, ey = o.y - x[j].y, ez = o.z - x[j].z, ew = o.w - x[j].w;
        pp[0] += 2.f * (o.x * x[j].x + o.y * x[j].y + o.z * x[j].z + o.w * x[j].w);
        pp[1] += 2.f * (ex * ex + ey * ey + ez * ez + ew * ew);
        if (ep.H) {
          const int r = row0 + rr;
          const float xs[4] = {x[j].x, x[j].y, x[j].z, x[j].w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int cc = c0 + cl + i;
            if (r < ep.M && cc < ep.M) {
              const double h = ep.h_f64 ? ((const double*)ep.H)[(size_t)r * ep.ldh + cc]
                                        : (double)((const float*)ep.H)[(size_t)r * ep.ldh + cc];
              pp[2] += 2.f * xs[i] * (float)h;
            }
          }
        }
        store_out4<BF16>(ep, off, o);
        *reinterpret_cast<float4*>(&tp[tp_idx(rr, cl)]) = o;
      }
    }
    __syncwarp();
    // mirror: eight lanes per original column, four consecutive rows each
    const int cs = lane >> 3, gr = lane & 7;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int cc = cs + 4 * j;
      const float4 m = make_float4(tp[tp_idx(4 * gr, cc)], tp[tp_idx(4 * gr + 1, cc)],
                                   tp[tp_idx(4 * gr + 2, cc)], tp[tp_idx(4 * gr + 3, cc)]);
      store_out4<BF16>(ep, (size_t)(c0 + cc) * Mp + row0 + 4 * gr, m);
    }
    __syncwarp();
  } else {
    // diagonal block: lane = column, element (row0 + k, c0 + lane)
    const int c = c0 + lane;
    float o[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const int r = row0 + k;
      const bool keep = c >= r;
      const bool on_diag = c == r && r < ep.M;
      const size_t off = (size_t)r * Mp + c;
      const float a = tp[tp_idx(k, lane)];
      const float x = ep.X[off];
      const float sg = fmaf(f2th, x, a * is2);
      // weight: an element above the diagonal stands for its mirror too
      const float w = keep ? (c == r ? 1.f : 2.f) : 0.f;
      const float e = sg - x - (on_diag ? thtb : 0.f);  // (S - D)_rc
      pp[0] += w * sg * x;
      pp[1] += w * e * e;
      if (on_diag) {
        dpart[0] += (double)x;
        dpart[1] += (double)sg;
      }
      if (ep.H && r < ep.M && c < ep.M) {
        const double h = ep.h_f64 ? ((const double*)ep.H)[(size_t)r * ep.ldh + c]
                                  : (double)((const float*)ep.H)[(size_t)r * ep.ldh + c];
        const float d = x + (on_diag ? thf : 0.f);
        pp[2] += w * d * (float)h;
      }
      o[k] = sg;
      if (keep) store_out1<BF16>(ep, off, sg);
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 32; ++k) tp[tp_idx(k, lane)] = o[k];
    __syncwarp();
    const int r = row0 + lane;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const int cc = c0 + k;
      if (cc <= r) continue;
      store_out1<BF16>(ep, (size_t)cc * Mp + r, tp[tp_idx(lane, k)]);
    }
    __syncwarp();
  }
}

// The epilogues run once per tile, so their code is fetched cold every
// time: each keeps one copy of its block body in a runtime loop over the
// four 32-column blocks and moves the block's accumulator registers to
// shared memory with this (a switch over the block gives every case
// compile-time register indices).
template <int P>
__device__ __forceinline__ void acc_to_tp(const float (&acc)[128], float* tp, int lane) {
#pragma unroll
  for (int g = 0; g < 8; ++g)
    *reinterpret_cast<float4*>(&tp[tp_idx(lane, 4 * g)]) =
        make_float4(acc[32 * P + 4 * g], acc[32 * P + 4 * g + 1], acc[32 * P + 4 * g + 2],
                    acc[32 * P + 4 * g + 3]);
}
// GEMM2 epilogue of one warp for one 32 x 32 block, laid out as in
// gemm1_block (the caller has written s^2 (X Sigma)_{row0+lane, c0+k} to
// row `lane` of `tp`): X_{n+1} = ca X + cb Sigma + cz Z (+ cj on the
// diagonal of the unpadded block) is formed with eight lanes per row, so the
// X and Sigma loads and the stores are whole row segments.  In a block of
// the diagonal 128-block only elements on or above the diagonal are stored
// (element-wise), those above it mirrored.  Without products (mma false)
// the block is a copy of X.
template <bool BF16>
__device__ __forceinline__ void gemm2_block(const Epi& ep, int row0, int c0, bool diag_blk,
                                            bool mma, float ca, float cb, float cj, float cz,
                                            float* tp) {
  const int lane = threadIdx.x & 31;
  const int Mp = ep.Mp;
  const float is2 = ep.inv_s2;
  const int rs = lane >> 3, cl = 4 * (lane & 7);
  const size_t cbase = (size_t)c0 + cl;
  float4 xx[8], ss[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const size_t off = (size_t)(row0 + rs + 4 * j) * Mp + cbase;
    xx[j] = *reinterpret_cast<const float4*>(ep.X + off);
    ss[j] = *reinterpret_cast<const float4*>(ep.Sig + off);
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int rr = rs + 4 * j;
    const size_t off = (size_t)(row0 + rr) * Mp + cbase;
    const float4 a = *reinterpret_cast<const float4*>(&tp[tp_idx(rr, cl)]);
    float4 o = xx[j];
    if (mma) {
      o.x = fmaf(ca, xx[j].x, fmaf(cb, ss[j].x, cz * (a.x * is2)));
      o.y = fmaf(ca, xx[j].y, fmaf(cb, ss[j].y, cz * (a.y * is2)));
      o.z = fmaf(ca, xx[j].z, fmaf(cb, ss[j].z, cz * (a.z * is2)));
      o.w = fmaf(ca, xx[j].w, fmaf(cb, ss[j].w, cz * (a.w * is2)));
    }
    if (!diag_blk) {
      store_out4<BF16>(ep, off, o);
    } else {
      const int r = row0 + rr;
      float ov[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int c = c0 + cl + i;
        if (mma && c == r && r < ep.M) ov[i] += cj;
        if (c >= r) store_out1<BF16>(ep, off + i, ov[i]);
      }
      o = make_float4(ov[0], ov[1], ov[2], ov[3]);
    }
    *reinterpret_cast<float4*>(&tp[tp_idx(rr, cl)]) = o;
  }
  __syncwarp();
  const int cs = lane >> 3, gr = lane & 7;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int cc = cs + 4 * j;
    const float4 m = make_float4(tp[tp_idx(4 * gr, cc)], tp[tp_idx(4 * gr + 1, cc)],
                                 tp[tp_idx(4 * gr + 2, cc)], tp[tp_idx(4 * gr + 3, cc)]);
    const size_t mo = (size_t)(c0 + cc) * Mp + row0 + 4 * gr;
    if (!diag_blk) {
      store_out4<BF16>(ep, mo, m);
    } else {
      const float mv[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (c0 + cc > row0 + 4 * gr + i) store_out1<BF16>(ep, mo + i, mv[i]);
    }
  }
  __syncwarp();
}

// Everything one tile needs: its block coordinates, operand maps, the
// epilogue pointers of its instance and the update coefficients.
struct TileCtx {
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
  if (!BATCHED) {
    tc_tile(t, base.Mp / BM, base.Mp / BN, c.I, c.J);
    c.skip = false;
    c.ah = mAh;
    c.al = mAl;
    c.bh = mBh;
    c.bl = mBl;
  } else {
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
    tc_tile(t - it.tc_off, it.Mp / BM, it.Mp / BN, c.I, c.J);
  }
  const State* st = c.ep.st;
  c.mma = !c.skip && (MODE == 1 || st->apply != 0);
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
  if (!BATCHED) {
    State* st = ep.st;
    if (st->stopped || st->timeout) return;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t accf_bar[2];
  __shared__ __align__(8) uint64_t acce_bar[2];
  __shared__ __align__(8) uint64_t fin_bar;
  __shared__ uint32_t tmem_holder;
  __shared__ double red[2 * 8 * 5];
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
  int* timeout_flag = BATCHED ? &items[0].st->timeout : &ep.st->timeout;

  if (warp < 4) {
    reg_dealloc<kCtlRegs>();
    if (warp == 0 && lane == 0) {
      // ---------------- TMA producer ----------------
      uint32_t g = 0;  // global stage counter
      bool alive = true;
      for (int t = blockIdx.x; t < ep.ntiles && alive; t += gridDim.x) {
        TileCtx c;
        make_ctx<MODE, BATCHED>(t, ep, &mAh, &mAl, &mBh, &mBl, items, tile_inst, c);
        for (int kb = 0; kb < c.nkb; ++kb, ++g) {
          const uint32_t s = g % STAGES;
          if (g >= STAGES && !mbar_wait(&empty_bar[s], ((g / STAGES) - 1) & 1)) {
            atomicOr(timeout_flag, 1);
            alive = false;
            break;
          }
          const uint32_t stage = sbase + s * kStageBytes;
          mbar_expect_tx(&full_bar[s], kStageBytes);
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
          tma_load_2d(ah, &full_bar[s], stage, kx, c.I * BM);
          tma_load_2d(al, &full_bar[s], stage + kABytes, kx, c.I * BM);
          tma_load_2d(bh, &full_bar[s], stage + 2 * kABytes, kx, c.J * BN);
          tma_load_2d(bh, &full_bar[s], stage + 2 * kABytes + kBBytes / 2, kx, c.J * BN + 128);
          tma_load_2d(bl, &full_bar[s], stage + 2 * kABytes + kBBytes, kx, c.J * BN);
          tma_load_2d(bl, &full_bar[s], stage + 2 * kABytes + kBBytes + kBBytes / 2, kx,
                      c.J * BN + 128);
        }
      }
      // every issued load must land before the CTA exits
      const uint32_t first = g > STAGES ? g - STAGES : 0;
      for (uint32_t k = first; k < g; ++k)
        if (!mbar_wait(&full_bar[k % STAGES], (k / STAGES) & 1)) atomicOr(timeout_flag, 1);
    } else if (warp == 1 && lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t idesc = idesc_f16(BF16 ? 1 : 0);
      uint32_t g = 0, qc = 0;  // global stage and chunk counters
      bool alive = true;
      for (int t = blockIdx.x; t < ep.ntiles && alive; t += gridDim.x) {
        TileCtx c;
        make_ctx<MODE, BATCHED>(t, ep, &mAh, &mAl, &mBh, &mBl, items, tile_inst, c);
        const int nchunk = c.nkb / kc_stages<MODE>();
        for (int ch = 0; ch < nchunk && alive; ++ch, ++qc) {
          const uint32_t b = qc & 1;
          if (qc >= 2 && !mbar_wait(&acce_bar[b], ((qc >> 1) - 1) & 1)) {
            atomicOr(timeout_flag, 1);
            alive = false;
            break;
          }
          tc_fence_after();
          const uint32_t acc = tmem + b * 256;
          for (int ks = 0; ks < kc_stages<MODE>(); ++ks, ++g) {
            const uint32_t s = g % STAGES;
            if (!mbar_wait(&full_bar[s], (g / STAGES) & 1)) {
              atomicOr(timeout_flag, 1);
              alive = false;
              break;
            }
            tc_fence_after();
            const uint32_t a_h = sbase + s * kStageBytes;
            const uint32_t a_l = a_h + kABytes;
            const uint32_t b_h = a_h + 2 * kABytes;
            const uint32_t b_l = b_h + kBBytes;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint32_t off = kk * 32;  // 16 halves = 32 B inside the 64 B swizzle row
              const uint32_t first = (ks == 0 && kk == 0) ? 0u : 1u;
              umma(acc, sdesc(a_h + off), sdesc(b_h + off), idesc, first);
              umma(acc, sdesc(a_h + off), sdesc(b_l + off), idesc, 1u);
              umma(acc, sdesc(a_l + off), sdesc(b_h + off), idesc, 1u);
            }
            umma_commit(&empty_bar[s]);
          }
          umma_commit(&accf_bar[b]);
        }
      }
      // every MMA issued here must be complete before TMEM is freed
      umma_commit(&fin_bar);
      if (!mbar_wait(&fin_bar, 0)) atomicOr(timeout_flag, 1);
    }
  } else {
    reg_alloc<kDrainRegs>();
    // ---------------- drain + epilogue (warps 4..11) ----------------
    // TMEM lane quarter is fixed by the warp's rank within its warpgroup
    const int dw = warp - 4, q = warp & 3, half = dw >> 2;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    float* tp = reinterpret_cast<float*>(smem_raw + (sbase - raw) + STAGES * kStageBytes) +
                dw * 32 * 32;
    uint32_t qc = 0, nred = 0;
    bool alive = true;
    for (int t = blockIdx.x; t < ep.ntiles; t += gridDim.x) {
      TileCtx c;
      make_ctx<MODE, BATCHED>(t, ep, &mAh, &mAl, &mBh, &mBl, items, tile_inst, c);
      if (c.skip) continue;  // uniform over the CTA
      float acc[128];
#pragma unroll
      for (int k = 0; k < 128; ++k) acc[k] = 0.f;
      const int nchunk = c.nkb / kc_stages<MODE>();
      for (int ch = 0; ch < nchunk; ++ch, ++qc) {
        const uint32_t b = qc & 1;
        if (alive) {
          // warp-uniform: tcgen05.ld below is a warp-collective instruction
          const bool got = __all_sync(0xffffffffu, mbar_wait(&accf_bar[b], (qc >> 1) & 1));
          if (!got) {
            if (lane == 0) atomicOr(timeout_flag, 1);
            alive = false;
          }
        }
        if (!alive) break;
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
      // all drain warps agree on whether the tile completed
      drain_bar_sync();
      const bool ok = alive && !(*(volatile int*)timeout_flag);
      // GEMM1 partials: element sums in FP32 (per lane, then a float shuffle
      // tree), the diagonal sums Tr X, Tr Sigma in FP64 (dpart[0..1])
      double dpart[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      float pp[3] = {0.f, 0.f, 0.f};
      const int jb = 2 * c.J + half;
      if (ok && jb >= c.I) {
        if constexpr (MODE == 1) {
          const double th = c.ep.st->theta;
          const float thf = (float)th, f2th = (float)(2.0 * th), thtb = (float)(th * (1.0 - th));
#pragma unroll 1
          for (int part = 0; part < 4; ++part) {
            switch (part) {
              case 0: acc_to_tp<0>(acc, tp, lane); break;
              case 1: acc_to_tp<1>(acc, tp, lane); break;
              case 2: acc_to_tp<2>(acc, tp, lane); break;
              default: acc_to_tp<3>(acc, tp, lane); break;
            }
            gemm1_block<BF16>(c.ep, c.I * BM + 32 * q, c.J * BN + half * 128 + part * 32,
                              jb == c.I, thf, f2th, thtb, pp, dpart, tp);
          }
        } else if constexpr (MODE == 2) {
#pragma unroll 1
          for (int part = 0; part < 4; ++part) {
            switch (part) {
              case 0: acc_to_tp<0>(acc, tp, lane); break;
              case 1: acc_to_tp<1>(acc, tp, lane); break;
              case 2: acc_to_tp<2>(acc, tp, lane); break;
              default: acc_to_tp<3>(acc, tp, lane); break;
            }
            gemm2_block<BF16>(c.ep, c.I * BM + 32 * q, c.J * BN + half * 128 + part * 32,
                              jb == c.I, c.mma, c.ca, c.cb, c.cj, c.cz, tp);
          }
        } else if constexpr (MODE == 4) {
          const float inv = (float)(1.0 / (kRefScale * check_delta_scale(c.ep.st->R)));
          check_row(c.ep, c.I * BM + 32 * q + lane, c.J * BN + half * 128, jb == c.I, acc, inv,
                    pp, dpart);
        } else {
          refine_row(c.ep, c.I * BM + 32 * q + lane, c.J * BN + half * 128, jb == c.I, acc);
        }
      }
      if (MODE == 1 || MODE == 4) {
        // FP64 arithmetic is slow on this part: only warps on a diagonal
        // block (warp-uniform) reduce the FP64 sums, and six lanes of warp
        // 0 add the warps' rows of the table in parallel.  The table is
        // double-buffered by the count of reduced tiles, so one barrier per
        // tile suffices: a warp writes this buffer again only after the
        // next tile's barrier, which warp 0 reaches after reading it.
        const float s2 = warp_sum_f(pp[0]), s3 = warp_sum_f(pp[1]), s4 = warp_sum_f(pp[2]);
        double d0 = 0.0, d1 = 0.0;
        if (jb == c.I) {
          d0 = warp_sum(dpart[0]);
          d1 = warp_sum(dpart[1]);
        }
        double* r = red + (nred & 1) * 40;
        if (lane == 0) {
          r[dw * 5] = d0;
          r[dw * 5 + 1] = d1;
          r[dw * 5 + 2] = (double)s2;
          r[dw * 5 + 3] = (double)s3;
          r[dw * 5 + 4] = (double)s4;
        }
        drain_bar_sync();
        if (dw == 0 && lane < kPartFields) {
          double sacc = 0.0;
          if (lane < 5)
            for (int w = 0; w < 8; ++w) sacc += r[w * 5 + lane];
          ep.part[(size_t)t * kPartFields + lane] = sacc;
        }
        ++nred;
      }
      if (!ok) break;
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
  if (((uintptr_t)ptr & 15u) != 0 || ((size_t)Mp * 2) % 16 != 0 || Mp % BN != 0) {
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

template <int MODE, bool BF16, bool BATCHED>
int launch_tc(const TcOperands* A, const TcOperands* B, const Epi& ep, const BatchItem* items,
              const int* tile_inst, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<MODE, BF16, BATCHED>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_bytes<MODE>());
    if (e != cudaSuccess) return 1;
    // the register split must fit the pool the CTA is launched with, or
    // the drain warpgroups' setmaxnreg.inc would wait forever
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, tc_gemm_kernel<MODE, BF16, BATCHED>) != cudaSuccess ||
        fa.numRegs * kThreads < (int)(128 * kCtlRegs + 256 * kDrainRegs))
      return 1;
    attr = true;
  }
  const int grid = ep.ntiles < sm_count() ? ep.ntiles : sm_count();
  if (BATCHED) {
    CUtensorMap dummy;
    memset(&dummy, 0, sizeof dummy);
    tc_gemm_kernel<MODE, BF16, true><<<grid, kThreads, smem_bytes<MODE>(), s>>>(
        dummy, dummy, dummy, dummy, ep, items, tile_inst);
  } else {
    tc_gemm_kernel<MODE, BF16, false><<<grid, kThreads, smem_bytes<MODE>(), s>>>(A->hi, A->lo, B->hi, B->lo,
                                                                         ep, nullptr, nullptr);
  }
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 1;
}
}  // namespace

int tc_pad(int M) { return ((M + BN - 1) / BN) * BN; }

int tc_encode_map(void* map, const void* ptr, int Mp, int bf16, char* err, int errlen, int box_k) {
  return encode_map((CUtensorMap*)map, ptr, Mp, bf16, err, errlen, box_k);
}

int tc_num_tiles(int Mp) {
  const int NI = Mp / BM, NJ = Mp / BN;
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
                    float split_scale, int* /*dev_err*/, cudaStream_t s) {
  Epi ep{};
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
                    float split_scale, int* /*dev_err*/, cudaStream_t s) {
  Epi ep{};
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
                        const double* dscale, int M, int Mp, State* st, cudaStream_t s) {
  Epi ep{};
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
                    cudaStream_t s) {
  Epi ep{};
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

size_t tc_map_bytes() { return 6 * sizeof(CUtensorMap); }

// Host images of the six tensor maps of one batched instance.
int tc_build_batch_maps(void* maps_host, const BatchItem& it, int bf16, char* err, int errlen) {
  CUtensorMap* m = (CUtensorMap*)maps_host;
  const void* ptrs[6] = {it.Xh[0], it.Xl[0], it.Xh[1], it.Xl[1], it.Sh, it.Sl};
  for (int k = 0; k < 6; ++k)
    if (encode_map(&m[k], ptrs[k], it.Mp, bf16, err, errlen)) return 1;
  return 0;
}

int tc_launch_batch_gemm(int mode, const BatchItem* items, int batch, const int* tile_inst,
                         int ntiles, double* part, int bf16, float split_scale, cudaStream_t s) {
  (void)batch;
  Epi ep{};
  ep.part = part;
  ep.ntiles = ntiles;
  ep.split_scale = split_scale;
  ep.inv_s2 = 1.0f / (split_scale * split_scale);
  if (mode == 1)
    return bf16 ? launch_tc<1, true, true>(nullptr, nullptr, ep, items, tile_inst, s)
                : launch_tc<1, false, true>(nullptr, nullptr, ep, items, tile_inst, s);
  if (mode == 3) {
    // refinement product: fp16 halves, scales carried by the operands
    ep.split_scale = 1.0f;
    ep.inv_s2 = 1.0f;
    return launch_tc<3, false, true>(nullptr, nullptr, ep, items, tile_inst, s);
  }
  return bf16 ? launch_tc<2, true, true>(nullptr, nullptr, ep, items, tile_inst, s)
              : launch_tc<2, false, true>(nullptr, nullptr, ep, items, tile_inst, s);
}

}  // namespace gcp
