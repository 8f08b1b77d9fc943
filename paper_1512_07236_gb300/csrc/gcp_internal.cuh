// Internal declarations shared by the translation units of libgcp.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gcp.h"

namespace gcp {

constexpr double kU64 = 1.1102230246251565e-16;  // 2^-53

// Device-resident solver state.  One instance per solve; written only by
// the single-block control kernels, read by every kernel of an iteration.
struct State {
  int n;            // steps applied so far (all phases)
  int n_lowp;       // steps applied in the split-precision phase
  int stopped;      // 1 once the current phase has stopped
  int status;       // gcp_status
  int apply;        // the GEMM2 of this iteration applies an update
  int parity;       // index of the ping-pong buffer holding the current iterate
  int phase;        // 1 = split precision, 0 = FP64
  int lowp_done;    // split-precision phase finished (stagnated or converged)
  int no_gap;
  int timeout;      // a bounded wait in a kernel gave up
  int hist_n;
  int converged;    // the stop test held
  int terminal;     // stopped for good (max_iter, stagnation, hard error)
  int n_phase0;     // n when the current phase began
  int split_floor;  // fixed-iteration split phase: the products stalled,
                    // every further step is an identity step
  double c, a, b;           // c_n and the polynomial coefficients of D_{n+1}
  double T1, T2, T3, R, E;  // traces of the last evaluated iterate
  double Rp0, Rp1;          // residuals of the two previous evaluated iterates
  double mu, beta2, hmin, hmax, theta;
  double xshift;            // J coefficient of X+ (split phase)
  double g3;                // D^3 coefficient of the step (-2 for HPCP)
  double alpha;             // mixing coefficient of the guess (Eq. hpcpguess)
};

// Scalar options every control kernel needs (passed by value).
struct Ctl {
  int M, N;
  int stop;         // gcp_stop
  int max_iter;
  int fixed_iters;
  int hist_cap;
  int phase;        // 1 split precision, 0 FP64
  int final_phase;  // this phase decides the final status
  int endgame;      // McWeeny endgame (split and refinement phases only)
  int mcw_only;     // every step is a McWeeny step (exact-slice refinement)
  int method;       // gcp_method
  int phase_max;    // > 0: at most this many steps in this phase
  double tol;
  double u;         // unit roundoff of the phase's state (den guard)
  // fixed-iteration split phase: per step, how c_n was taken (kStep*), for
  // the adjoint; may be null
  int* step_kind;
};

// How a step of the fixed-iteration split phase took c_n.
constexpr int kStepIdentity = 0;   // no update (0/0 guard or stalled products)
constexpr int kStepRestoring = 1;  // Eq. hpcp3, c_n = (num + (Tr D - N)/2) / den
constexpr int kStepMcWeeny = 2;    // Eq. hpcp3 with c_n = 1/2 (Eq. mcweeny3)

// Number of partial-sum fields written per GEMM1 tile.
constexpr int kPartFields = 6;  // T1, T2, T3, R^2, E, spare

// Digit slices of the exact-slice refinement and the scale of its fp16
// operand halves (gcp_ozaki.cu).
constexpr int kOzSlices = 9;
constexpr double kRefScale = 16384.0;  // 2^14
// Scale of Delta = D1 - D in the stop-test product after a refinement step:
// 2^(13 - e) with 2^e > 2 R, R = ||D^2 - D||_F of the iterate before the
// step; D1 - D = X((1 - a) I - 2D), |a| <= 0.1, so |Delta_ij| <= 1.2 R and
// the scaled entries stay below 2^13.
__host__ __device__ inline double check_delta_scale(double R) {
  int e = 0;
  frexp(2.0 * R, &e);  // 2 R < 2^e
  return ldexp(1.0, 13 - e);
}

// Per-instance descriptor of a batched solve (device memory).  Every
// instance has its own state, buffers and slices of the batched work lists.
// The iterate buffer in use is State::parity: GEMM1 reads buffer `parity`;
// the control kernel flips it when it schedules an update, so GEMM2 reads
// `parity ^ 1` and writes `parity`.
struct BatchItem {
  State* st;
  const void* H;
  void* D_out;
  float* X[2];
  void* Xh[2];
  void* Xl[2];
  float* Sig;
  void* Sh;
  void* Sl;
  double* D64[2];
  double* S64;
  const void* maps;  // 6 tensor maps: X0 hi, X0 lo, X1 hi, X1 lo, Sigma hi, Sigma lo
  int M, Mp, N, ld, ldd;
  int tc_off, tc_n;    // tensor-core tiles in the batched work list
  int f64_off, f64_n;  // FP64 tiles in the batched work list
  int gblocks;         // reduction blocks of the guess/energy passes
                       // (guess_partial_blocks(M): the single-solve layout)
  // exact-slice refinement (mixed modes): digit slices, row scales of D and
  // of X = S - D, fp16 halves of both, and 15 tensor maps (the 9 slices with
  // 64-wide boxes, then D hi, D lo, X hi, X lo, slice 0 and slice 1 with
  // 32-wide boxes: the operands of the stop-test product)
  void* oz_sl[kOzSlices];
  double* oz_rs;
  double* oz_xs;
  void *oz_dh, *oz_dl, *oz_xh, *oz_xl;
  const void* oz_maps;
  int oz_off;  // first partial-sum slot (oz_finalize_blocks(M) slots, as a single solve)
};

// ---- guess (gcp_guess.cu) ------------------------------------------------
int guess_partial_blocks(int M);
// Per-block partials of the guess reduction: min_i(H_ii - r_i),
// max_i(H_ii + r_i), Tr H, max|H_ii|, sum_{i != j} H_ij^2.
constexpr int kGuessFields = 5;
void launch_guess_reduce(const void* H, int h_f64, int M, int ld, double* part, cudaStream_t s);
// Combine partials into mu, theta and the coefficient b of the guess
// (gcp_guess mode; the HPCP+ search reads the diagonal of H), into State.
void launch_guess_finalize(const double* part, int nblocks, int M, int N, const void* H,
                           int h_f64, int ld, int guess_mode, State* st, cudaStream_t s);
// max_{i<j} |H_ij - H_ji| and max_ij |H_ij| into out[0], out[1] (device,
// zeroed here first).
void launch_sym_check(const void* H, int h_f64, int M, int ld, double* out, cudaStream_t s);
// D0 = theta I + beta2 (mu I - H) (FP64 or FP32 out), padded area zero.
void launch_guess_write_d(const void* H, int h_f64, int M, int ld, void* D, int d_f64, int ldd,
                          int rows_pad, const State* st, cudaStream_t s);
// X0 = D0 - theta J in FP32 plus its split halves (fp16 or bf16), Mp x Mp.
void launch_guess_write_x(const void* H, int h_f64, int M, int ld, float* X, void* Xh, void* Xl,
                          int Mp, int bf16, float split_scale, const State* st, cudaStream_t s);

// ---- FP64 products (gcp_fp64.cu) -------------------------------------------
int f64_tile(int M);
int f64_num_tiles(int M);
// S = D D over upper tiles, mirrored; epilogue partials per tile.
void launch_f64_gemm1(const double* D, double* S, int M, int ld, const void* H, int h_f64, int ldh,
                      double* part, const State* st, cudaStream_t s);
// Dn = a D + b S + g3 S D over upper tiles, mirrored (a, b, g3 from State).
void launch_f64_gemm2(const double* S, const double* D, double* Dn, int M, int ld,
                      const State* st, cudaStream_t s);

// ---- control (gcp_control.cu) --------------------------------------------
void launch_control(const double* part, int ntiles, State* st, double* hist, Ctl ctl,
                    unsigned long long cond_handle, int use_cond, cudaStream_t s);
// Stop test after a refinement step from the check product's partials
// (Tr D1, Tr D1^2, -, R1^2): stops the phase, converged, when R1 <= tol.
void launch_check_control(const double* part, int ntiles, State* st, double* hist, Ctl ctl,
                          unsigned long long cond_handle, int use_cond, cudaStream_t s);
void launch_state_init(State* st, int phase, cudaStream_t s);
void launch_phase_begin(State* st, int phase, cudaStream_t s);
// D_out = buf[parity] converted to the output dtype (FP64 source).
void launch_copy_out_f64(const double* buf0, const double* buf1, const State* st, int M, int ld,
                         void* out, int out_f64, int ldo, cudaStream_t s);
// D_out = theta J + X[parity] (FP32 source, shifted).
void launch_copy_out_x(const float* X0, const float* X1, const State* st, int M, int ldx,
                       void* out, int out_f64, int ldo, cudaStream_t s);
// D64 = theta J + X[parity] (upper triangle mirrored).
void launch_x_to_d64(const float* X0, const float* X1, State* st, int M, int ldx, double* D,
                     int ldd, cudaStream_t s);
// E = sum_ij D_ij H_ij into State::E (per-block partials in `part`).
void launch_energy(const void* D, int d_f64, int ldd, const void* H, int h_f64, int ldh, int M,
                   double* part, State* st, cudaStream_t s);
// Generic conversions for gcp_step.
void launch_d_to_x(const void* D, int d_f64, int M, int ld, float* X, void* Xh, void* Xl, int Mp,
                   int bf16, float split_scale, double theta, cudaStream_t s);
void launch_fill(const void* val_src_unused, void* out, int out_f64, int M, int ldo, double diag,
                 cudaStream_t s);
void launch_convert(const void* in, int in_f64, int ldi, void* out, int out_f64, int ldo, int M,
                    cudaStream_t s);

// ---- tensor-core split products (gcp_tc.cu) -----------------------------
struct TcOperands;  // opaque: tensor maps for one (hi, lo) pair
int tc_pad(int M);
int tc_num_tiles(int Mp);
// Tensor map (CUtensorMap) of an Mp x Mp 16-bit row-major operand, boxes of
// 128 rows x box_k columns: box_k = 32 with 64-byte swizzle, 64 with
// 128-byte swizzle.
int tc_encode_map(void* map, const void* ptr, int Mp, int bf16, char* err, int errlen,
                  int box_k = 32);
// Build tensor maps for a pair of split halves (Mp x Mp, row-major).
int tc_make_operands(TcOperands** op, const void* hi, const void* lo, int Mp, int bf16,
                     char* err, int errlen);
void tc_free_operands(TcOperands* op);
// Mode 1: Y = X X, Sigma = 2 theta X + Y, partials.  Mode 2: Z = X Sigma,
// X+ update.  See gcp_tc.cu for the epilogue formulas.
// Every tensor-core launch takes `scratch`, tc_scratch_bytes() of device
// memory: the drain warps hand each finished tile to the epilogue warps
// through two 128 x 256 FP32 slots per CTA.
size_t tc_scratch_bytes();
// wait_ns: bound of every device-side wait (0: the default 2 s); stall: a
// diagnostic that makes the drain wait on a barrier nobody arrives on, so
// that every role of the kernel runs into its bound (gcp_debug_timeout).
int tc_launch_gemm1(const TcOperands* opX, const float* X, float* Sig, void* Sh, void* Sl,
                    int M, int Mp, const void* H, int h_f64, int ldh, double* part, State* st,
                    int bf16, float split_scale, float* scratch, cudaStream_t s,
                    unsigned long long wait_ns = 0, int stall = 0);
int tc_launch_gemm2(const TcOperands* opS, const TcOperands* opX, const float* X, const float* Sig,
                    float* Xn, void* Xnh, void* Xnl, int M, int Mp, State* st, int bf16,
                    float split_scale, float* scratch, cudaStream_t s);
void tc_set_smem_attrs();
// Refinement step (FP64): Dn = S - 2 Z - a (S - D) with Z = X D from the
// fp16 halves of X = S - D (opX, row i scaled by xscale_i) and of D (opD,
// row j scaled by kRefScale / dscale_j), and a = State::a (0 for the
// McWeeny step).
int tc_launch_mcweeny64(const TcOperands* opX, const TcOperands* opD, const double* S64,
                        const double* D64, double* Dn64, const double* xscale,
                        const double* dscale, int M, int Mp, State* st, float* scratch,
                        cudaStream_t s);
// W = D1^2 - D^2 from the halves of D (opD, scale kRefScale), of
// Delta = D1 - D (opDelta, scale check_delta_scale(R)) and of Delta at the
// scale kRefScale (emaps, device maps), and the per-tile partials of
// D1^2 - D1 = S + W - D1.
int tc_launch_check(const TcOperands* opD, const TcOperands* opDelta, const void* emaps,
                    const double* S64, const double* D1, double* part, int M, int Mp, State* st,
                    float* scratch, cudaStream_t s);
// Plain product C = inv_scale (A B) of two split-fp16 operands (Mp x Mp;
// the kernel computes A B^T, so B is given as the rows of B^T), FP32 out:
// over all tiles, or (symmetric != 0: the result is known to be symmetric)
// the upper tiles with the lower triangle mirrored.  st: a state with
// stopped = 0 (its timeout flag records a wait that gave up).
int tc_launch_product(const TcOperands* A, const TcOperands* B, float* C, int Mp, int symmetric,
                      float inv_scale, State* st, float* scratch, cudaStream_t s);
// Device copies (cudaMalloc'ed, freed with cudaFree) of the hi/lo tensor
// maps of a pair of Mp x Mp fp16 arrays, for operands named through memory.
int tc_make_device_maps(void** dev, const void* hi, const void* lo, int Mp, char* err,
                        int errlen);

// ---- exact slice products (gcp_ozaki.cu) ---------------------------------
// D (FP64, M x M) -> per-row scale 2^e_i with |D_ij| <= 2^e_i / 2, nine
// signed base-32 digit slices (fp16, Mp x Mp) and the fp16 halves of
// kRefScale D_ij / 2^e_i (the D operand of the refinement product).
struct OzOperands;  // opaque: tensor maps of the nine slices
int oz_make_operands(OzOperands** op, void* const* slices, int Mp, char* err, int errlen);
void oz_free_operands(OzOperands* op);
void launch_oz_slice(const double* D, int M, int Mp, void* const* slices, double* rscale,
                     void* Dh, void* Dl, const State* st, cudaStream_t s);
// S = D D up to the slicing (FP64 out, M x M, both triangles): digit-pair
// weights up to wcap (<= 0: all), see oz_weight_cap.
int launch_oz_gemm(const OzOperands* op, const double* rscale, double* S64, int M, int Mp,
                   int wcap, State* st, cudaStream_t s);
// Highest digit-pair weight a refinement with stop tolerance tol needs, the
// estimate of what the dropped weights add to ||D^2 - D||_F (0 with all
// weights), and the number of digit-pair products of a plan.
int oz_weight_cap(int M, double tol);
double oz_tail_estimate(int M, double tol);
int oz_num_products(int M, int wcap);
// Partials (Tr D, Tr S, sum S o D, ||S - D||^2, 0) per block for the control
// kernel, and the fp16 halves of xscale_i X_ij, X = S - D, with a power of
// two xscale_i per row (max_j |xscale_i X_ij| < 2^13).
// Blocks of the finalize pass (eight rows at a time, one warp each), and so
// its partial-sum slots: single solves and every instance of a batch alike.
__host__ __device__ inline int oz_finalize_blocks(int M) {
  const int b = (M + 7) / 8;
  return b < 1024 ? b : 1024;
}
// fp16 halves (Mp x Mp, zero padded) of kRefScale D, of s Delta with
// s = check_delta_scale(State::R) and of kRefScale Delta, Delta = D1 - D.
void launch_check_halves(const double* D64, const double* D1, int M, int Mp, void* Dh, void* Dl,
                         void* Xh, void* Xl, void* Eh, void* El, const State* st,
                         cudaStream_t s);
void launch_oz_finalize(double* S64, const double* D64, int M, int Mp, double* part,
                        void* Xh, void* Xl, double* xscale, const State* st, cudaStream_t s);
// Digit bits b and slice count of the slicing for an M-long inner dimension.
int oz_digit_bits(int M);
int oz_num_slices(int M);
// Batched forms over the instances' BatchItem (work list: the tensor-core
// tiles), reading and writing the current iterate D64[State::parity].
void launch_batch_oz_slice(const BatchItem* items, int batch, int maxM, cudaStream_t s);
int launch_batch_oz_gemm(const BatchItem* items, const int* tile_inst, int ntiles, int maxM,
                         int wcap, cudaStream_t s);
void launch_batch_oz_finalize(const BatchItem* items, int batch, int maxM, double* part,
                              cudaStream_t s);
// Operands of the batched stop-test product (as launch_check_halves per
// instance: D = D64[parity ^ 1], D1 = D64[parity]).
void launch_batch_check_halves(const BatchItem* items, int batch, int maxM, cudaStream_t s);
size_t oz_batch_map_bytes();
int oz_build_batch_maps(void* maps_host, const BatchItem& it, char* err, int errlen);

// ---- adjoint (gcp_adjoint.cu) --------------------------------------------
constexpr double kU32 = 5.9604644775390625e-08;  // 2^-24
// guess: gcp_guess of the forward; method: gcp_method of its steps.
int adjoint_backward(void** ws, const void* H, int M, int N, int ld, int h_f64, int guess,
                     int method, const void* GD, double gE, void* dLdH, int K, int ck,
                     double* D64_0, double* D64_1, double* S64, double* part, double* gpart,
                     State* st, double* hist, cudaStream_t s, char* err, int errlen);
void adjoint_free(void* ws);
// Coefficients (a, b, g3) of one step D+ = a D + b D^2 + g3 D^3 and their
// derivatives with respect to c_n.
struct StepCoeffs {
  double a, b, g3, da, db, dg3;
};
StepCoeffs step_coeffs(double c, int method);
// The guess part of the adjoint: dL/dH from G0 = dL/dD_0 and D_K (FP64,
// M x M), written to dLdH (ld, h dtype); guess: gcp_guess.
int adjoint_guess(const void* H, int M, int N, int ld, int h_f64, int guess, const double* G0,
                  const double* DK, double gE, void* dLdH, double* gpart, State* st,
                  cudaStream_t s, char* err, int errlen);
// The same derivative with the iterates in the split state and the
// products on the tensor cores (FP32, HPCP steps; gcp_adjoint_tc.cu).
// scratch: tc_scratch_bytes() for the tensor-core kernels; hist: >= K + 2
// records.
int adjoint_backward_tc(void** ws, const void* H, int M, int N, int ld, int h_f64, int guess,
                        const void* GD, double gE, void* dLdH, int K, int ck, State* st,
                        double* part, double* gpart, double* hist, float* scratch,
                        cudaStream_t s, char* err, int errlen);
void adjoint_tc_free(void* ws);

// ---- batched solves (many instances per launch) --------------------------
// guess: per-instance Gershgorin/trace partials (gstride slots of 4 doubles
// per instance in `gpart`, the instance using its own gblocks of them, in
// the same order as a single solve), parameters into each State, then D0/X0.
void launch_batch_guess(const BatchItem* items, int batch, int maxM, int h_f64, int split,
                        int bf16, float split_scale, double* gpart, int gstride, int guess_mode,
                        cudaStream_t s);
void launch_batch_control(const double* part, const BatchItem* items, int batch, Ctl ctl,
                          cudaStream_t s);
// Stop test after a batched refinement step from the check product's tile
// partials of each instance (as launch_check_control of a single solve).
void launch_batch_check_control(const double* part, const BatchItem* items, int batch, Ctl ctl,
                                cudaStream_t s);
void launch_batch_any_active(const BatchItem* items, int batch, unsigned long long cond,
                             int use_cond, int* active_out, cudaStream_t s);
void launch_batch_state_init(const BatchItem* items, int batch, int phase, cudaStream_t s);
void launch_batch_phase_begin(const BatchItem* items, int batch, int phase, cudaStream_t s);
void launch_batch_x_to_d64(const BatchItem* items, int batch, int maxM, cudaStream_t s);
void launch_batch_copy_out(const BatchItem* items, int batch, int maxM, int from_x, int out_f64,
                           cudaStream_t s);
void launch_batch_energy(const BatchItem* items, int batch, int out_f64, int h_f64, double* gpart,
                         int gstride, cudaStream_t s);
// FP64 products over the work list of all instances (32 x 32 tiles).
int batch_f64_tiles(int M);
void launch_batch_f64_gemm1(const BatchItem* items, int batch, const int* tile_inst, int ntiles,
                            double* part, cudaStream_t s);
void launch_batch_f64_gemm2(const BatchItem* items, int batch, const int* tile_inst, int ntiles,
                            cudaStream_t s);
// Tensor-core products over the work list of all instances.
int tc_build_batch_maps(void* maps_host, const BatchItem& it, int bf16, char* err, int errlen);
size_t tc_map_bytes();
// `order`: the order in which the CTAs take the work list's tiles (null: the
// list's own); results do not depend on it.
int tc_launch_batch_gemm(int mode, const BatchItem* items, int batch, const int* tile_inst,
                         const int* order, int ntiles, double* part, int bf16, float split_scale,
                         float* scratch, cudaStream_t s);
// Estimated cost of tile `local` of an Mp x Mp instance's work list, in
// units of one 32 x 32 block's epilogue: 2 for a block above the diagonal
// (direct and mirrored stores), 1 for a diagonal block, plus Mp / 128 for the
// products.
int tc_tile_cost(int Mp, int local);

}  // namespace gcp
