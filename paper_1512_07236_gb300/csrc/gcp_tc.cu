// Split-precision tensor-core products of one GCP step (sm_103a: tcgen05 +
// TMEM + TMA), with the step's elementwise work fused into the epilogues.
//
// State.  The iterate is held shifted, X = D - theta J (J = identity on the
// unpadded M x M block), in FP32, plus two 16-bit halves of s*X
// (s = split scale, a power of two):
//   fp16: h = rn(sX), l = rn((sX - h) 2^11)     sX ~ h + 2^-11 l
//   bf16: h = rn(sX), l = rn(sX - h)            sX ~ h + l
// Early in the recursion D is close to theta I, so X is small and the
// rounding of the state and of the products is relative to |X|, not to
// |D|: the shift costs nothing (Tr D = N fixes theta) and keeps the
// subspace of the final projector from being rotated by rounding while the
// occupied and virtual eigenvalues of D are still close together.
//
// Products.  A * B^T with both operands K-major; since every operand is
// symmetric, B = B^T.  Per K block three MMAs accumulate in TMEM (FP32):
//   acc0 += Ah Bh,   acc1 += Ah Bl + Al Bh,   AB ~ (acc0 + w_lo acc1) / s^2
// (the lo*lo term is below the FP32 accumulator's resolution).
//
// GEMM1 (Y = X X).  With S = D^2 = theta^2 J + Sigma, Sigma = 2 theta X + Y,
// the epilogue writes Sigma (FP32 + halves, both triangles) and per-tile
// partial sums Tr X, Tr Sigma, sum Sigma o X, ||S - D||_F^2 (elementwise,
// S - D = Sigma - X - theta(1-theta) J) and optionally sum D o H, from which
// the control kernel forms Tr D, Tr D^2, Tr D^3 (Eq. mcwgamb).
// GEMM2 (Z = X Sigma).  D_{n+1} = a D + b S - 2 D S with a = 1 - 2c,
// b = 2 + 2c (Eq. hpcp3) becomes, for X_{n+1} = D_{n+1} - theta J,
//   X_{n+1} = 2 theta (1-theta)(theta - c) J + (a - 2 theta^2) X
//             + (b - 2 theta) Sigma - 2 Z.
//
// Schedule.  One CTA computes a 128 x 256 tile (two 128 x 128 blocks) of
// the upper block triangle; blocks below the diagonal inside a tile are
// skipped in the epilogue, off-diagonal blocks are also stored mirrored.
// Warp 0 lane 0 issues TMA loads (SWIZZLE_128B, 64-wide K blocks, a
// 2-stage ring of 96 KB stages), warp 1 lane 0 issues tcgen05.mma, all
// four warps run the epilogue from TMEM (warp w owns lanes 32w..32w+31).
// Every mbarrier wait is bounded (2 s); on expiry the kernel records
// State::timeout, skips the rest and still frees its TMEM.
#include <cuda.h>
#include <stdio.h>

#include "gcp_device.cuh"
#include "gcp_internal.cuh"

namespace gcp {

struct TcOperands {
  CUtensorMap hi;
  CUtensorMap lo;
};

namespace {
constexpr int BM = 128, BN = 256, BK = 64, STAGES = 2;
constexpr int kTcThreads = 128;
constexpr uint32_t kABytes = BM * BK * 2;                     // 16 KB
constexpr uint32_t kBBytes = BN * BK * 2;                     // 32 KB
constexpr uint32_t kStageBytes = 2 * kABytes + 2 * kBBytes;  // 96 KB
constexpr uint32_t kSmemBytes = STAGES * kStageBytes + 1024;
constexpr uint32_t kTmemCols = 512;  // acc0: cols [0,256), acc1: [256,512)
constexpr unsigned long long kWaitNs = 2000000000ull;

struct Epi {
  const float* X;    // current shifted iterate (FP32, Mp x Mp)
  const float* Sig;  // Sigma (mode 2)
  float* out;        // Sigma (mode 1) or X_{n+1} (mode 2), FP32
  void* out_h;       // split halves of `out`
  void* out_l;
  const void* H;     // optional, for sum D o H (mode 1)
  int h_f64, ldh;
  double* part;      // per-tile partials (mode 1)
  State* st;
  int M, Mp;
  float split_scale;    // s
  float inv_s2;         // 1/s^2
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on the phase of `bar` with the given parity.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (true) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (gtimer() - t0 > kWaitNs) return false;
  }
}
__device__ __forceinline__ void tma_load_2d(const CUtensorMap* map, uint64_t* bar, void* dst, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
// Shared-memory matrix descriptor: K-major, SWIZZLE_128B, 8-row groups
// 1024 B apart (SBO), descriptor version 1 (bits 46-47).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;              // LBO (ignored for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // SBO
  d |= (uint64_t)1 << 46;              // version
  d |= (uint64_t)2 << 61;              // SWIZZLE_128B
  return d;
}
// Instruction descriptor, kind::f16: D fp32 (bits 4-5 = 1), A/B format
// (bits 7-9, 10-12: 0 fp16, 1 bf16), both K-major, N>>3 at bit 17,
// M>>4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f16(int bf16) {
  return (1u << 4) | ((uint32_t)bf16 << 7) | ((uint32_t)bf16 << 10) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                     uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Linear tile index -> (I, J): I a 128-row block, J a 256-column block,
// kept when the tile reaches the upper block triangle (2J + 1 >= I).
// Column-block-major order so that consecutive CTAs share their B panel.
__device__ __forceinline__ void tc_tile(int t, int NI, int NJ, int& I, int& J) {
  int j = 0;
  while (true) {
    const int cnt = (2 * j + 2 < NI ? 2 * j + 2 : NI);  // I in [0, min(2J+2, NI))
    if (t < cnt) {
      I = t;
      J = j;
      return;
    }
    t -= cnt;
    ++j;
    if (j >= NJ) {  // unreachable for valid t
      I = 0;
      J = 0;
      return;
    }
  }
}

template <int MODE, bool BF16>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                   const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
                   const Epi ep) {
  using HT = typename Split<BF16>::T;
  State* st = ep.st;
  if (st->stopped || st->timeout) return;
  const int NI = ep.Mp / BM, NJ = ep.Mp / BN;
  int I, J;
  tc_tile(blockIdx.x, NI, NJ, I, J);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = I * BM + warp * 32 + lane;  // this thread's output row
  const bool do_mma = (MODE == 1) || st->apply;
  const int Mp = ep.Mp;

  // Epilogue coefficients.
  const double th = st->theta;
  const float f2th = (float)(2.0 * th);
  const float thtb = (float)(th * (1.0 - th));
  float ca = 0.f, cb = 0.f, cj = 0.f;
  if (MODE == 2) {
    ca = (float)(st->a - 2.0 * th * th);
    cb = (float)(st->b - 2.0 * th);
    cj = (float)st->xshift;
  }
  const float lo_w = Split<BF16>::kLoWeight;

  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t acc_bar;
  __shared__ uint32_t tmem_holder;
  __shared__ double red[32 * 5];
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  uint8_t* sptr = smem_raw + (sbase - raw);

  uint32_t tmem = 0;
  bool ok = true;
  if (do_mma) {
    if (threadIdx.x == 0) {
      for (int s = 0; s < STAGES; ++s) {
        mbar_init(&full_bar[s], 1);
        mbar_init(&empty_bar[s], 1);
      }
      mbar_init(&acc_bar, 1);
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
    tmem = tmem_holder;

    const int nk = Mp / BK;
    if (warp == 0 && lane == 0) {
      // TMA producer
      int issued = 0;
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES, it = kb / STAGES;
        if (kb >= STAGES && !mbar_wait(&empty_bar[s], (it - 1) & 1)) {
          atomicOr(&st->timeout, 1);
          break;
        }
        uint8_t* stage = sptr + s * kStageBytes;
        mbar_expect_tx(&full_bar[s], kStageBytes);
        const int kx = kb * BK;
        tma_load_2d(&mAh, &full_bar[s], stage, kx, I * BM);
        tma_load_2d(&mAl, &full_bar[s], stage + kABytes, kx, I * BM);
        tma_load_2d(&mBh, &full_bar[s], stage + 2 * kABytes, kx, J * BN);
        tma_load_2d(&mBh, &full_bar[s], stage + 2 * kABytes + kBBytes / 2, kx, J * BN + 128);
        tma_load_2d(&mBl, &full_bar[s], stage + 2 * kABytes + kBBytes, kx, J * BN);
        tma_load_2d(&mBl, &full_bar[s], stage + 2 * kABytes + kBBytes + kBBytes / 2, kx,
                    J * BN + 128);
        issued = kb + 1;
      }
      // drain: every issued load must have landed before the CTA can exit
      for (int kb = issued - STAGES < 0 ? 0 : issued - STAGES; kb < issued; ++kb) {
        if (!mbar_wait(&full_bar[kb % STAGES], (kb / STAGES) & 1)) atomicOr(&st->timeout, 1);
      }
    } else if (warp == 1 && lane == 0) {
      // MMA issuer
      const uint32_t idesc = idesc_f16(BF16 ? 1 : 0);
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES, it = kb / STAGES;
        if (!mbar_wait(&full_bar[s], it & 1)) {
          atomicOr(&st->timeout, 1);
          break;
        }
        tc_fence_after();
        const uint32_t a_h = sbase + s * kStageBytes;
        const uint32_t a_l = a_h + kABytes;
        const uint32_t b_h = a_h + 2 * kABytes;
        const uint32_t b_l = b_h + kBBytes;
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint32_t off = kk * 32;  // 16 halves = 32 B inside the 128 B swizzle row
          const uint32_t acc = (kb | kk) ? 1u : 0u;
          umma(tmem, sdesc(a_h + off), sdesc(b_h + off), idesc, acc);
          umma(tmem + 256, sdesc(a_h + off), sdesc(b_l + off), idesc, acc);
          umma(tmem + 256, sdesc(a_l + off), sdesc(b_h + off), idesc, 1u);
        }
        umma_commit(&empty_bar[s]);
      }
      umma_commit(&acc_bar);
    }
    __syncwarp();
    bool mine = mbar_wait(&acc_bar, 0);
    if (!mine) atomicOr(&st->timeout, 1);
    tc_fence_after();
    // CTA-uniform decision: tcgen05.ld below must run in every warp or none
    ok = __syncthreads_and(mine && !(*(volatile int*)&st->timeout)) != 0;
  }

  // ---------------- epilogue ----------------
  double dpart[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const bool in_m = row < ep.M;
  if (ok) {
#pragma unroll 1
    for (int ch = 0; ch < BN / 16; ++ch) {
      const int c0 = J * BN + ch * 16;
      const int jb = c0 / BM;
      if (jb < I) continue;  // block below the diagonal: its mirror is computed elsewhere
      const bool diag_blk = (jb == I);
      float acc0[16], acc1[16];
      if (do_mma) {
        const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + ch * 16;
        tmem_ld16(ta, acc0);
        tmem_ld16(ta + 256, acc1);
        tmem_ld_wait();
      } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) acc0[k] = acc1[k] = 0.f;
      }
      const size_t rowoff = (size_t)row * Mp + c0;
      float x[16];
      {
        const float4* px = reinterpret_cast<const float4*>(ep.X + rowoff);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 t = px[q];
          x[4 * q] = t.x;
          x[4 * q + 1] = t.y;
          x[4 * q + 2] = t.z;
          x[4 * q + 3] = t.w;
        }
      }
      float o[16];
      if (MODE == 1) {
        float p2 = 0.f, p3 = 0.f, p4 = 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const float y = (acc0[k] + lo_w * acc1[k]) * ep.inv_s2;
          const float sg = fmaf(f2th, x[k], y);  // Sigma = 2 theta X + Y
          o[k] = sg;
          const int c = c0 + k;
          // weight: an element above the diagonal stands for its mirror too;
          // in a diagonal block only the upper triangle is kept
          const float w = diag_blk ? (c > row ? 2.f : (c == row ? 1.f : 0.f)) : 2.f;
          const bool on_diag = diag_blk && (c == row) && in_m;
          const float e = sg - x[k] - (on_diag ? thtb : 0.f);  // (S - D)_ij
          p2 = fmaf(w * sg, x[k], p2);
          p3 = fmaf(w * e, e, p3);
          if (on_diag) {
            dpart[0] += (double)x[k];
            dpart[1] += (double)sg;
          }
          if (ep.H && in_m && c < ep.M) {
            const double h = ep.h_f64 ? ((const double*)ep.H)[(size_t)row * ep.ldh + c]
                                      : (double)((const float*)ep.H)[(size_t)row * ep.ldh + c];
            const float d = x[k] + (on_diag ? (float)th : 0.f);
            p4 = fmaf(w * d, (float)h, p4);
          }
        }
        dpart[2] += (double)p2;
        dpart[3] += (double)p3;
        dpart[4] += (double)p4;
      } else {
        float sg[16];
        const float4* ps = reinterpret_cast<const float4*>(ep.Sig + rowoff);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 t = ps[q];
          sg[4 * q] = t.x;
          sg[4 * q + 1] = t.y;
          sg[4 * q + 2] = t.z;
          sg[4 * q + 3] = t.w;
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          if (do_mma) {
            const float z = (acc0[k] + lo_w * acc1[k]) * ep.inv_s2;
            const bool on_diag = diag_blk && (c0 + k == row) && in_m;
            o[k] = fmaf(ca, x[k], fmaf(cb, sg[k], -2.f * z)) + (on_diag ? cj : 0.f);
          } else {
            o[k] = x[k];
          }
        }
      }
      // stores: FP32 + halves.  The result is made exactly symmetric: in a
      // diagonal block only elements on or above the diagonal are written,
      // each also to its mirror position.
      HT h[16], l[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) Split<BF16>::split(o[k] * ep.split_scale, h[k], l[k]);
      if (diag_blk) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int c = c0 + k;
          if (c < row) continue;
          const size_t d0 = (size_t)row * Mp + c, mo = (size_t)c * Mp + row;
          ep.out[d0] = o[k];
          reinterpret_cast<HT*>(ep.out_h)[d0] = h[k];
          reinterpret_cast<HT*>(ep.out_l)[d0] = l[k];
          if (c > row) {
            ep.out[mo] = o[k];
            reinterpret_cast<HT*>(ep.out_h)[mo] = h[k];
            reinterpret_cast<HT*>(ep.out_l)[mo] = l[k];
          }
        }
      } else {
        float4* po = reinterpret_cast<float4*>(ep.out + rowoff);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          po[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
        uint4* ph = reinterpret_cast<uint4*>(reinterpret_cast<HT*>(ep.out_h) + rowoff);
        uint4* pl = reinterpret_cast<uint4*>(reinterpret_cast<HT*>(ep.out_l) + rowoff);
        ph[0] = *reinterpret_cast<const uint4*>(&h[0]);
        ph[1] = *reinterpret_cast<const uint4*>(&h[8]);
        pl[0] = *reinterpret_cast<const uint4*>(&l[0]);
        pl[1] = *reinterpret_cast<const uint4*>(&l[8]);
        // mirror: element (row, c) -> (c, row); lanes hold consecutive rows,
        // so each of these stores is one coalesced segment per warp
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const size_t mo = (size_t)(c0 + k) * Mp + row;
          ep.out[mo] = o[k];
          reinterpret_cast<HT*>(ep.out_h)[mo] = h[k];
          reinterpret_cast<HT*>(ep.out_l)[mo] = l[k];
        }
      }
    }
  }
  if (MODE == 1) {
    block_sum<5>(dpart, red);
    if (threadIdx.x == 0) {
      double* p = ep.part + (size_t)blockIdx.x * kPartFields;
      p[0] = dpart[0];
      p[1] = dpart[1];
      p[2] = dpart[2];
      p[3] = dpart[3];
      p[4] = dpart[4];
      p[5] = 0.0;
    }
  }
  if (do_mma) {
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"(kTmemCols));
    }
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

int encode_map(CUtensorMap* m, const void* ptr, int Mp, int bf16, char* err, int errlen) {
  EncodeTiledFn enc = get_encode(err, errlen);
  if (!enc) return 1;
  if (((uintptr_t)ptr & 15u) != 0 || ((size_t)Mp * 2) % 16 != 0 || Mp % BN != 0) {
    snprintf(err, errlen, "tensor map: misaligned operand or size");
    return 1;
  }
  cuuint64_t dims[2] = {(cuuint64_t)Mp, (cuuint64_t)Mp};
  cuuint64_t strides[1] = {(cuuint64_t)Mp * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                   const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    snprintf(err, errlen, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return 1;
  }
  return 0;
}

template <int MODE, bool BF16>
int launch_tc(const TcOperands* A, const TcOperands* B, const Epi& ep, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<MODE, BF16>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return 1;
    attr = true;
  }
  const int nt = tc_num_tiles(ep.Mp);
  tc_gemm_kernel<MODE, BF16><<<nt, kTcThreads, kSmemBytes, s>>>(A->hi, A->lo, B->hi, B->lo, ep);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : 1;
}
}  // namespace

int tc_pad(int M) { return ((M + BN - 1) / BN) * BN; }

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
  ep.split_scale = split_scale;
  ep.inv_s2 = 1.0f / (split_scale * split_scale);
  return bf16 ? launch_tc<1, true>(opX, opX, ep, s) : launch_tc<1, false>(opX, opX, ep, s);
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
  ep.split_scale = split_scale;
  ep.inv_s2 = 1.0f / (split_scale * split_scale);
  return bf16 ? launch_tc<2, true>(opX, opS, ep, s) : launch_tc<2, false>(opX, opS, ep, s);
}

void tc_set_smem_attrs() {}

}  // namespace gcp
