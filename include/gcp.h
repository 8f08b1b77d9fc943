/*
 * gcp.h -- C ABI of libgcp: generalized canonical purification (GCP, the
 * paper's hole-particle canonical purification, HPCP) on one GB300 GPU.
 *
 * Problem (paper's problem statement, Eq. mcw4a with the footnote on
 * orthonormal bases): given a real symmetric Hamiltonian H (M x M, in an
 * orthonormal basis) and an electron count 0 <= N <= M, return the
 * idempotent density matrix D (D^2 = D) with Tr D = N that minimises
 * E = Tr(H D), without diagonalising H.
 *
 * Method:
 *   guess   D_0 = beta_1 I + beta_2 (mu I - H)                 (Eq. dmguess)
 *           beta_1 = theta = N/M, mu = Tr H / M,
 *           beta_2 = min{theta/(H_max - mu), (1-theta)/(mu - H_min)},
 *           H_min/H_max Gershgorin bounds                      (Eq. pmcpguess)
 *   step    c_n = Tr(D^2 - D^3) / Tr(D - D^2)                   (Eq. mcwgamb)
 *           D_{n+1} = D + 2 (D^2 (I-D) - c_n D (I-D))           (Eq. hpcp3)
 *                   = (1-2c) D + (2+2c) D^2 - 2 D^3
 *   stop    ||D^2 - D||_F <= tol, or Tr(D (I-D)) <= tol (the paper's test,
 *           text after Eq. hpcp3)
 *   energy  E = Tr(H D)
 *
 * Conventions for every entry point:
 *   - Matrix arguments are DEVICE pointers owned by the caller, row-major
 *     with leading dimension `ld` (elements, ld >= M).  Because every matrix
 *     here is symmetric, row- and column-major are the same; H is read in
 *     full and must be symmetric (it is not checked).
 *   - `dtype` arguments take gcp_dtype: GCP_F64 (double) or GCP_F32 (float).
 *   - Small outputs (gcp_result, the info arrays) are HOST pointers, written
 *     after the call has synchronised its stream.  Every call here is
 *     synchronous at exit with respect to `opt->stream`.
 *   - The handle owns all workspace (device memory, graphs, tensor maps);
 *     workspace grows on demand and is released by gcp_destroy.  A handle
 *     must not be used from two host threads at once.
 *   - Errors are returned as gcp_status and never abort the process.
 *     GCP_ERR_NOT_CONVERGED still fills D_out and the result.
 *     gcp_last_error() gives a one-line description of the last failure.
 */
#ifndef GCP_H_
#define GCP_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GCP_OK = 0,
  GCP_ERR_INVALID_ARG = 1,     /* bad pointer, size, dtype or option */
  GCP_ERR_NOT_CONVERGED = 2,   /* max_iter reached or stagnated above tol */
  GCP_ERR_ILL_CONDITIONED = 3, /* c_0 outside [0,1]: Eqs. pmcpcons2-3 violated */
  GCP_ERR_NO_GAP = 4,          /* H = mu I: zero-width Gershgorin interval */
  GCP_ERR_NONFINITE = 5,       /* NaN/Inf in a trace */
  GCP_ERR_TIMEOUT = 6,         /* a bounded device-side wait gave up */
  GCP_ERR_CUDA = 7,            /* a CUDA runtime/driver call failed */
  GCP_ERR_UNSUPPORTED = 8,     /* combination not built */
  GCP_ERR_NO_CHECKPOINT = 9    /* gcp_backward without a matching forward */
} gcp_status;

typedef enum { GCP_F64 = 0, GCP_F32 = 1 } gcp_dtype;

/* Arithmetic of the matrix products.
 *   GCP_FP64        FP64 products (SIMT DFMA) and FP64 state throughout.
 *   GCP_FP16X3      split-FP16 tensor-core products (tcgen05, FP32
 *                   accumulation in TMEM, 3 products per GEMM) on the
 *                   shifted state X = D - theta I held in FP32; stops at
 *                   its own accuracy floor.
 *   GCP_BF16X3      as FP16X3 with BF16 halves.
 *   GCP_MIXED_FP16  FP16X3 until the residual stagnates, then refinement
 *                   steps in FP64 arithmetic until the stop test holds
 *                   (gcp_options.refine picks how their products run).
 *   GCP_MIXED_BF16  BF16X3 bulk, the same refinement.  Its subspace error
 *                   (about 1e-5 at M = 8192, gap 0.01) is ten times that of
 *                   GCP_MIXED_FP16: the 8-bit bf16 halves carry 16 bits of X.
 *   GCP_MIXED_AUTO  picks the arithmetic from the problem: GCP_FP64 when
 *                   M < 512 (the tensor-core tiles are mostly padding there
 *                   and the FP64 products are cheap) or tol < 1e-10 (below
 *                   the floor of the exact-slice refinement at large M),
 *                   GCP_MIXED_FP16 otherwise.  The gap of H, the other
 *                   factor in the subspace error of the split phase, is not
 *                   known before the solve.  gcp_result reports what ran
 *                   (iters_lowp > 0 for the mixed path).
 *   GCP_FP32        an FP32 state with split-FP16 tensor-core products: for
 *                   gcp_solve the arithmetic of GCP_FP16X3; for
 *                   gcp_backward the tensor-core adjoint (forward, segment
 *                   recomputation and the adjoint's three products per step
 *                   on the tensor cores, FP32 elementwise work).
 *                   Fixed-iteration split solves (the recursion
 *                   gcp_backward differentiates) take c_n as a free-running
 *                   split solve does: Eq. mcwgamb with the rounding drift of
 *                   Tr D absorbed (Tr D_{n+1} = N), the McWeeny step once
 *                   ||D^2 - D||_F < 0.05; where a free-running solve would
 *                   stop at the floor of its products, the remaining steps
 *                   are identity steps.                                     */
typedef enum {
  GCP_FP64 = 0,
  GCP_FP16X3 = 1,
  GCP_BF16X3 = 2,
  GCP_MIXED_FP16 = 3,
  GCP_MIXED_BF16 = 4,
  GCP_MIXED_AUTO = 5,
  GCP_FP32 = 6
} gcp_precision;

typedef enum {
  GCP_STOP_IDEMP_FRO = 0,  /* ||D^2 - D||_F <= tol (computed elementwise) */
  GCP_STOP_TRACE_DDBAR = 1 /* Tr(D - D^2) <= tol (the paper's test) */
} gcp_stop;

typedef struct {
  int prec;            /* gcp_precision (default GCP_FP64) */
  int stop;            /* gcp_stop (default GCP_STOP_IDEMP_FRO) */
  double tol;          /* stop tolerance (default 1e-12) */
  int max_iter;        /* cap on steps (default 100) */
  int fixed_iters;     /* > 0: run exactly this many steps, no stop test;
                          steps past the 0/0 guard (split precisions: or
                          past the floor of the products) become identity
                          steps */
  int ckpt_every;      /* checkpoint interval for gcp_backward (default 8) */
  int history_cap;     /* > 0: record up to this many per-step records */
  int use_graph;       /* 1 (default): device-side loop in one CUDA graph;
                          0: host-driven loop (debugging) */
  void* stream;        /* cudaStream_t; NULL = legacy default stream */
  int refine;          /* mixed modes, refinement products: 0 (default) exact
                          digit-slice products on the tensor cores with
                          McWeeny steps (M <= 29000, no fixed_iters;
                          gcp_solve and gcp_solve_batched);  1 FP64 SIMT
                          products and HPCP steps (always used otherwise) */
  int guess;           /* gcp_guess (default GCP_GUESS_CANONICAL) */
  int method;          /* gcp_method (default GCP_METHOD_HPCP) */
  int refine_iters;    /* mixed modes: at most this many refinement steps
                          (0, the default: only max_iter bounds them); a
                          solve that hits the cap without meeting tol returns
                          GCP_ERR_NOT_CONVERGED with the last iterate */
  int check_symmetry;  /* 1: before solving, measure max_ij |H_ij - H_ji| and
                          return GCP_ERR_INVALID_ARG when it exceeds
                          sym_tol * max_ij |H_ij| (default 0: not checked;
                          the split-precision paths read only the upper
                          triangle of H, the FP64 path all of it) */
  double sym_tol;      /* relative bound of the symmetry check (default 0:
                          exact symmetry) */
} gcp_options;

/* Initial guess.
 *   GCP_GUESS_CANONICAL  Eq. dmguess with the coefficients of Eq. pmcpguess:
 *                        D0 = theta I + beta_min (mu I - H).
 *   GCP_GUESS_HPCP_PLUS  Eq. hpcpguess, D0 = alpha D0_canonical +
 *                        (1 - alpha)(I - Dbar0) with the hole guess
 *                        Dbar0 = thetabar I - beta_max (mu I - H); alpha in
 *                        [0, 1] from Eq. hpcpguessalpha with delta = 2/3:
 *                        Tr D0^2 = N - delta N if theta <= 1/3,
 *                        N - delta (M - N) if theta >= 2/3, alpha = 1/2
 *                        otherwise.  Equivalently D0 = theta I + b (mu I - H),
 *                        b = alpha beta_min + (1 - alpha) beta_max.
 *   GCP_GUESS_HOLE       I - Dbar0 (alpha = 0): purifying it is the hole
 *                        purification of the paper (Eq. hpcp3 on Dbar), by
 *                        the particle-hole duality of the recursion.  Its
 *                        spectrum leaves [0, 1] away from half filling,
 *                        where the solve reports GCP_ERR_ILL_CONDITIONED.
 * gcp_backward differentiates all three. */
typedef enum {
  GCP_GUESS_CANONICAL = 0,
  GCP_GUESS_HPCP_PLUS = 1,
  GCP_GUESS_HOLE = 2
} gcp_guess;

/* Recursion.
 *   GCP_METHOD_HPCP  Eq. hpcp3: D+ = (1-2c) D + (2+2c) D^2 - 2 D^3.
 *   GCP_METHOD_PMCP  the canonical purification of Appendix A, Eq. pm1:
 *                    c <= 1/2: D+ = [(1-2c) D + (1+c) D^2 - D^3] / (1-c),
 *                    c >  1/2: D+ = [(1+c) D^2 - D^3] / c,
 *                    same c_n (Eq. mcwgamb).
 * Both conserve Tr D.  The refinement steps of the mixed modes are the
 * McWeeny step with the trace-restoring c for either method.  gcp_backward
 * differentiates both (GCP_METHOD_PMCP with GCP_FP64). */
typedef enum { GCP_METHOD_HPCP = 0, GCP_METHOD_PMCP = 1 } gcp_method;

typedef struct {
  int status;        /* gcp_status of the solve */
  int iters;         /* steps applied (all phases) */
  int iters_lowp;    /* steps applied in the split-precision phase */
  int iters_fp64;    /* steps applied in FP64 */
  double trace;      /* Tr D of the returned D (FP64 sum) */
  double energy;     /* E = Tr(H D) of the returned D */
  double idem_fro;   /* ||D^2 - D||_F at the last evaluated iterate (after an
                        exact-slice refinement step accepted by the stop-test
                        product: ||S + W - D1||_F, S = D^2 exact, W = D1^2 - D^2
                        from a split product; ~1e-7 of the step's residual) */
  double trace_ddbar;/* Tr(D - D^2) at the last evaluated iterate */
  double c_last;     /* last c_n used */
  double mu, beta2, hmin, hmax; /* guess parameters (Eq. pmcpguess); beta2 is
                                   the coefficient b actually used */
  double alpha;      /* mixing coefficient of Eq. hpcpguess (1 = canonical) */
} gcp_result;

/* Per-step record written when history_cap > 0 (gcp_get_history):
 * {n, T1 = Tr D, T2 = Tr D^2, T3 = Tr D^3, R = ||D^2-D||_F, c_n, E_n, phase}
 * phase: 0 = FP64, 1 = split precision.  c_n is NaN on the final record. */
#define GCP_HISTORY_FIELDS 8

void gcp_default_options(gcp_options* opt);
const char* gcp_status_string(int status);

gcp_status gcp_create(void** handle);
gcp_status gcp_destroy(void* handle);
const char* gcp_last_error(void* handle);

/* Canonical initial guess (Eq. dmguess, Eq. pmcpguess).
 * H: device, M x M, ld, h_dtype.  D0: device, M x M, ldd, d_dtype (written).
 * info (host, 5 doubles, may be NULL): mu, beta2, H_min, H_max, theta.
 * Returns GCP_ERR_NO_GAP (D0 = theta I) when the Gershgorin interval has
 * zero width.  0 < N < M required (the trivial fillings have no guess). */
gcp_status gcp_init_guess(void* handle, const void* H, int M, int N, int ld, int h_dtype,
                          void* D0, int ldd, int d_dtype, double* info,
                          const gcp_options* opt);

/* One step of Eq. hpcp3 in place on D (device, M x M, ld, d_dtype), in the
 * arithmetic opt->prec selects (GCP_FP64 requires d_dtype GCP_F64; the
 * split-precision modes take GCP_F32 and theta = N/M for the shift).
 * out (host, 6 doubles, may be NULL): T1, T2, T3, R = ||D^2 - D||_F, c, and
 * 1.0 if the update was applied (0.0 when Tr(D - D^2) was at the 0/0 guard). */
gcp_status gcp_step(void* handle, void* D, int M, int N, int ld, int d_dtype, double* out,
                    const gcp_options* opt);

/* Full solve: guess, recursion with device-side stop test, energy.
 * H: device, M x M, ld, h_dtype.  D_out: device, M x M, ldd, d_dtype.
 * res: host (may be NULL).  N = 0 and N = M return D = 0 / D = I. */
gcp_status gcp_solve(void* handle, const void* H, int M, int N, int ld, int h_dtype,
                     void* D_out, int ldd, int d_dtype, gcp_result* res,
                     const gcp_options* opt);

/* Copy the history of the last gcp_solve (host buffer, cap records of
 * GCP_HISTORY_FIELDS doubles); *n_out = records written. */
gcp_status gcp_get_history(void* handle, double* out, int cap, int* n_out);

/* Many independent solves of uneven size in one call (the same recursion and
 * readings as gcp_solve, applied to each instance).  H[b], D_out[b]: device
 * pointers (host arrays of `batch` pointers); H[b] is M[b] x M[b] with
 * leading dimension ld[b], D_out[b] is dense M[b] x M[b] (leading dimension
 * M[b]); M, N, ld: host arrays of length batch; all H in h_dtype and all D in
 * d_dtype.  res: host array of `batch` results (may be NULL).  Every kernel
 * of a step is one launch over the tiles of all instances; each instance has
 * its own c_n, stop test and status, and a stopped instance adds no work.
 * history_cap must be 0.  Returns the first non-OK instance status. */
gcp_status gcp_solve_batched(void* handle, int batch, const void* const* H, const int* M,
                             const int* N, const int* ld, int h_dtype, void* const* D_out,
                             int d_dtype, gcp_result* res, const gcp_options* opt);

/* Work order of the batched tensor-core products (scheduling only, no
 * counterpart in the paper).  In split-precision batched solves the CTAs
 * take the tiles of all instances' products from one work list; the first
 * solve for a given set of instance sizes (with at least two tiles per SM)
 * times the first step's GEMM1 under four candidate orders and keeps the
 * fastest for later solves of those sizes on this handle: 0 = instance after
 * instance, 1 = tiles by estimated cost, largest first, dealt to the CTAs in
 * turn, 2 = as 1 with every other round dealt in reverse, 3 = instance after
 * instance, largest instance first.  Results are the same under every
 * order, bit for bit.
 *
 * gcp_set_batched_order: order = -1 (default) times the candidates; 0, 1,
 * 2 or 3 fixes that candidate without timing.  GCP_ERR_INVALID_ARG
 * otherwise.  gcp_batched_order: *choice = the order the last
 * split-precision batched solve used; ms (4 doubles, may be NULL) = the
 * GEMM1 time of each candidate in milliseconds, -1 where none was timed
 * (fewer tiles, or a fixed order).  Host-only; no device work. */
gcp_status gcp_set_batched_order(void* handle, int order);
gcp_status gcp_batched_order(void* handle, int* choice, double* ms);

/* Reverse-mode derivative of L = <G_D, D_K> + g_E * Tr(H D_K), where D_K is
 * the iterate after exactly opt->fixed_iters steps of Eq. hpcp3 from the
 * guess of H (Eq. dmguess, Eq. pmcpguess); c_n depends on D_n (Eq. mcwgamb)
 * and the adjoint includes that dependence.  opt->prec: GCP_FP64 (FP64
 * iterates and products) or GCP_FP32 (the iterates of a GCP_FP32
 * fixed-iteration solve, products on the tensor cores; the derivative of
 * that computed recursion).
 * H: device M x M (ld, h_dtype); G_D: device M x M (ld, h_dtype) or NULL
 * (D_K is symmetric, so only the symmetric part of G_D matters);
 * dL_dH: device M x M (ld, h_dtype), written, symmetric (the derivative with
 * respect to a symmetric H; the Gershgorin bound contributes a subgradient).
 * opt->guess: any gcp_guess (the HPCP+ guess through its alpha, Eq.
 * hpcpguessalpha); opt->method: GCP_METHOD_HPCP or GCP_METHOD_PMCP (Eq. pm1;
 * GCP_FP64 only, GCP_ERR_UNSUPPORTED with GCP_FP32).
 * Runs the forward pass itself, keeping a checkpoint every opt->ckpt_every
 * steps (default 8) and recomputing the iterates in between; steps past the
 * 0/0 guard are identity steps.  0 < N < M required. */
gcp_status gcp_backward(void* handle, const void* H, int M, int N, int ld, int h_dtype,
                        const void* G_D, double g_E, void* dL_dH, const gcp_options* opt);

/* Allocation-free FP64 solve (the paper has no counterpart: this is a
 * deployment variant of gcp_solve).  For callers that must not allocate
 * device memory while solving -- a program whose memory pool already holds
 * the GPU's memory, a latency-bound loop that cannot take the implicit device
 * synchronisation of cudaMalloc/cudaFree, or code that cannot keep a handle.
 * Same arguments and FP64 arithmetic as gcp_solve with opt->prec = GCP_FP64
 * (other precisions and history return GCP_ERR_UNSUPPORTED), but no handle:
 * the workspace is one fixed file-scope device array of 6.3 MB, so
 * M <= 512 (larger M returns GCP_ERR_INVALID_ARG with a message in err).
 * The array is shared by every call on a device and keeps the previous
 * call's contents; calls whose GPU work overlaps race on it, so order them.
 * The first call on a device looks up the array's device address.  The
 * step loop is driven from the host (a state read and a stream
 * synchronisation after every step), so the call is synchronous and must not
 * be made while its stream is being captured into a CUDA graph.
 * GCP_MIXED_AUTO runs this FP64 path.  A loop that ends without the stop
 * test returns GCP_ERR_NOT_CONVERGED.  err (host, may be NULL): errlen bytes
 * for a one-line message. */
gcp_status gcp_solve_noalloc(const void* H, int M, int N, int ld, int h_dtype, void* D_out,
                             int ldd, int d_dtype, gcp_result* res, const gcp_options* opt,
                             char* err, int errlen);

/* Diagnostic (no counterpart in the paper): exercise the bounded waits of the
 * tensor-core kernel.  Launches one split-precision GEMM1 of size M on the
 * workspace of this handle with every device-side wait bounded by wait_s
 * seconds (0 < wait_s <= 10), after making its drain warps first wait on a
 * barrier that no thread arrives on: every role of the kernel reaches its
 * bound, records the timeout and returns (TMEM freed, context usable).
 * Returns GCP_ERR_TIMEOUT when the kernel reported it, which is the expected
 * result, GCP_OK if it did not.  The workspace contents are overwritten: a
 * following gcp_solve on the handle starts afresh. */
gcp_status gcp_debug_timeout(void* handle, int M, double wait_s, const gcp_options* opt);

/* Diagnostic (no counterpart in the paper): time the two products of one
 * step on the workspace left by the last gcp_solve on this handle (same M;
 * `prec` GCP_FP64 times the FP64 kernels, GCP_FP16X3/GCP_BF16X3 the
 * tensor-core ones and needs a prior split or mixed solve, GCP_MIXED_FP16
 * or GCP_MIXED_BF16 the products of an exact-slice refinement step -- the
 * digit-slice D^2, the fp16 split (D^2 - D) D and the stop-test product
 * W = D1^2 - D^2 -- and needs a prior mixed solve that used that
 * refinement; the slice product keeps the digit pairs a solve with
 * opt->tol keeps).  Each kernel is launched `reps` times on opt->stream,
 * bracketed by CUDA events; ms (host; 2 doubles, 4 for GCP_MIXED_*)
 * receives the mean duration of each product in milliseconds, and for
 * GCP_MIXED_* ms[3] the number of digit-pair products of the slice product.
 * The workspace iterate is overwritten: solve again before reading
 * results. */
gcp_status gcp_time_kernels(void* handle, int M, int N, int prec, int reps, double* ms,
                            const gcp_options* opt);

#ifdef __cplusplus
}
#endif
#endif /* GCP_H_ */
