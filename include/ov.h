/*
 * ov.h -- C ABI of the GB300 (sm_103a) contour-integral overlap library.
 *
 * The library computes, on one GPU,
 *
 *   sgn(H_W) b  ~=  S_N b = c0 b + sum_{j=1..N} c_j (z_j - H_W)^-1 b      (Eqs. 5-7)
 *   D_ov(m_q) b  =  (1 + m_q)/2 b + (1 - m_q)/2 gamma5 S_N b              (Eq. 1)
 *
 * for the hermitian Wilson-Dirac operator H_W = gamma5 D_W(-m0) (Eq. 1 and the
 * definition of H_W after it) on a 4D periodic lattice with SU(3) links, where
 * the nodes z_j and coefficients c_j come from the N-point trapezoid rule on an
 * ellipse (Eq. 7).  The resolvents (z_j - H_W)^-1 b of Eq. 6 are produced by one
 * shifted Krylov solve for all nodes at once (the shift-solver remark after
 * Eq. 7).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * dims = {Lx, Ly, Lz, Lt}; direction mu = 0,1,2,3 is x,y,z,t.
 * D_W psi(x) = (4r + m) psi(x) - 1/2 sum_mu [ (r - g_mu) U_mu(x) psi(x+mu)
 *                                            + (r + g_mu) U_mu(x-mu)^dag psi(x-mu) ],
 * m = -m0; r must be 1.  Space is periodic; time is periodic (bc_t = +1) or
 * antiperiodic (bc_t = -1, a sign on every hop across the t boundary).
 * Chiral basis: g_k = [[0, -i s_k], [i s_k, 0]] (k = x, y, z), g_t = [[0, 1], [1, 0]],
 * gamma5 = g_x g_y g_z g_t = diag(1, 1, -1, -1).
 *
 * Canonical layouts (all complex numbers interleaved re, im; x fastest):
 *   gauge field  U[mu][t][z][y][x][row 3][col 3]                 complex double
 *   spinor       psi[rhs][t][z][y][x][spin 4][colour 3]          complex double or float
 *   link force   F[mu][t][z][y][x][a 8]                          double (real)
 * V = Lx*Ly*Lz*Lt sites; one spinor is 12 V complex numbers.
 *
 * Ownership and streams: every vector argument is a pointer the caller owns and
 * keeps alive until the work enqueued on `stream` has finished.  Pointers are
 * DEVICE pointers unless the entry point or an option says otherwise.  `stream`
 * is a cudaStream_t passed as void* (NULL = the legacy default stream).  The
 * context owns its gauge copies, contour and workspace; workspace grows on
 * demand and is reused.  A context is not thread safe: serialise calls on it.
 *
 * Errors: every entry point returns an ov_status.  Nothing aborts, traps or
 * spins without bound on the device: every device loop has an iteration limit
 * and reports through the status.  ov_last_error() gives a one-line reason.
 */
#ifndef OV_H_
#define OV_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ov_ctx ov_ctx;

typedef enum {
  OV_OK = 0,
  OV_ERR_INVALID_ARG = 1,   /* bad pointer, size, flag or parameter            */
  OV_ERR_OUT_OF_MEMORY = 2, /* device allocation failed                        */
  OV_ERR_NOT_CONVERGED = 3, /* iteration limit hit; output holds the last iterate */
  OV_ERR_BREAKDOWN = 4,     /* a Krylov recurrence produced a non-finite scalar */
  OV_ERR_CUDA = 5,          /* a CUDA runtime call failed                      */
  OV_ERR_NO_GAUGE = 6,      /* ov_set_gauge has not been called                */
  OV_ERR_NO_CONTOUR = 7,    /* no contour set on the context                   */
  OV_ERR_SCRATCH_TOO_SMALL = 8 /* ov_apply_HW_noalloc: the call needs more than its fixed scratch */
} ov_status;

typedef enum { OV_FP64 = 0, OV_FP32 = 1 } ov_precision;

/* Solver modes for ov_sgn_HW_apply / ov_overlap_apply / ov_sgn_vjp. */
typedef enum {
  /* FP64 shifted solve: one Lanczos process on H_W serves every node; each node
   * keeps its own FP64 search direction and the weighted sum of Eq. 7 is
   * accumulated in the same pass (the paper's shift-solver structure). */
  OV_MODE_FP64 = 0,
  /* Mixed precision: FP32 shifted solve, then batched per-node FP64 true
   * residuals and FP32 defect-correction solves over all nodes x sources in
   * one multi-RHS launch, FP64 quadrature sum. */
  OV_MODE_MIXED = 1,
  /* FP64 coefficient-space Lanczos: the per-node recurrences of OV_MODE_FP64 are
   * carried out on the tridiagonal Lanczos matrix instead of on vectors, and the sum
   * of Eq. 7 becomes sum_i g_i v_i over the Lanczos basis.  The basis is kept in device
   * memory when min(max_iter, 1024) vectors per source fit a quarter of it (the sum is
   * then one read of the basis); otherwise a second Lanczos pass regenerates it.
   * Same result as OV_MODE_FP64 up to rounding; vector work independent of N. */
  OV_MODE_FP64_2PASS = 2,
  /* As OV_MODE_FP64_2PASS, always regenerating the basis (memory: three vectors per
   * source). */
  OV_MODE_FP64_REGEN = 3,
  /* As OV_MODE_FP64_2PASS with every vector operation -- the H_W stencil, the Lanczos
   * updates and the stored basis -- in FP32-pair (double-float) arithmetic on the FP32
   * units: each real is an unevaluated sum of two floats (~48-bit significand), sums
   * by error-free two-sum, products by FMA-based exact products.  Recurrence scalars,
   * inner products and the quadrature sum stay FP64.  All sources run in the same
   * launches.  Accuracy ~1e-13 relative; on GB300 (FP64 at 1/58 of the FP32 rate) it
   * replaces FP64 arithmetic in the bulk. */
  OV_MODE_F32X2 = 4
} ov_mode;

typedef enum {
  OV_CONTOUR_SINGLE = 0, /* sgn = 2 P_Gamma - 1, one ellipse around the positive spectrum */
  OV_CONTOUR_PAIR = 1    /* sgn = P_{Gamma+} - P_{Gamma-} (Eqs. 3, 5), centres +gamma and -gamma */
} ov_contour_form;

/* Options for the solves (pass NULL for the defaults in brackets). */
typedef struct {
  int mode;         /* ov_mode                                              [OV_MODE_FP64] */
  double tol;       /* per-node relative residual ||b - (z_j - H) y_j|| / ||b||   [1e-12] */
  int max_iter;     /* Krylov iteration limit per solve                          [20000] */
  int host_io;      /* 1: b / out / eta / grad_b are HOST pointers; copies to and
                       from the device are enqueued on `stream` inside the call
                       (page-locked inputs are read by a kernel, others copied)  [0] */
  int check_every;  /* iterations between host reads of the convergence flag  [32] */
  int use_graph;    /* 1: replay the per-iteration kernels from a CUDA graph     [1] */
  int node_chunk;   /* VJP: nodes whose forward and adjoint solutions are held at once;
                       0 = all.  Smaller values recompute the Krylov solve per chunk of
                       nodes: memory 2 x node_chunk x 12V complex doubles, work x chunks [0] */
} ov_solve_opts;

/* Per-call statistics (optional output, may be NULL). */
typedef struct {
  int iterations;        /* Krylov iterations of the (outer) solve, max over sources       */
  int refine_rounds;     /* OV_MODE_MIXED: defect-correction rounds                          */
  int inner_iterations;  /* OV_MODE_MIXED: total iterations of the correction solves          */
  int converged;         /* 1 if every node of every source met tol                           */
  double max_residual;   /* max over nodes and sources of the final relative residual          */
  double error_bound;    /* max over sources of sum_j |c_j| r_j / |Im z_j| (relative to ||b||):
                            bound on ||S_N b - out|| / ||b|| because ||(z - H)^-1|| <= 1/|Im z| */
  double ms;             /* wall time of the call on the host, milliseconds                  */
  double node_updates;   /* sum over iterations and sources of the nodes updated (the vector
                            work of the shifted solve is proportional to it)                 */
  double launches;       /* kernel launches the call enqueued (graph nodes included)          */
} ov_stats;

/* Spectral bounds from Lanczos (ov_place_contour). */
typedef struct {
  double lambda_min;     /* smallest Ritz value of H_W                                 */
  double lambda_max;     /* largest Ritz value of H_W                                   */
  double abs_max_bound;  /* upper bound on max |lambda| (Ritz value + residual bound)    */
  double gap;            /* estimate of min |lambda| (sqrt of the smallest Ritz value of H_W^2) */
  double predicted_error;/* max |r_N(lambda) - sgn(lambda)| over +-[gap, abs_max_bound] */
  double gamma, rho, alpha; /* the ellipse chosen                                       */
  int steps;             /* Lanczos steps taken                                          */
} ov_spectrum;

/* Create a context on CUDA device `device` for a lattice of size dims: the geometry,
 * boundary conditions, Wilson parameter r and mass -m0 of D_W(-m0) in Eq. 1 (the paper
 * fixes none of them; "Numerical experiments" uses m0 = 1 on 8^4).
 * bc_t: +1 periodic, -1 antiperiodic time.  r must be 1.0.  The context owns nothing
 * the caller passes later.
 * Errors: INVALID_ARG (dims < 1, V > 2^28, |bc_t| != 1, r != 1, m0 not finite), CUDA,
 * OUT_OF_MEMORY. */
int ov_create(ov_ctx** ctx, const int dims[4], int bc_t, double m0, double r, int device);

/* Release every device and host resource of the context (NULL is accepted).  Waits for
 * the context's outstanding work on the device first. */
int ov_destroy(ov_ctx* ctx);

/* One-line description of the last error on this context (never NULL; owned by the
 * context, valid until its next call). */
const char* ov_last_error(const ov_ctx* ctx);

/* Load the gauge field: the SU(3) links U_mu(x) of the Wilson operator D_W inside H_W
 * (Eq. 1; the paper's configurations are quenched SU(3) fields, "Numerical
 * experiments").  Canonical layout U[mu][t][z][y][x][3][3], V*4*9 complex doubles.
 * U may be a host (on_device = 0) or device (on_device = 1) pointer; it is copied on
 * `stream` and not retained.  The library keeps FP64, FP32 and double-float
 * structure-of-arrays copies.  Any cached contour placement is invalidated (explicit
 * contours are kept).  Errors: INVALID_ARG (null U), OUT_OF_MEMORY, CUDA. */
int ov_set_gauge(ov_ctx* ctx, const double* U, int on_device, void* stream);

/* out = H_W in (Eq. 1 and the definition of H_W = gamma5 D_W(-m0) after it) for nrhs
 * spinors in the canonical layout psi[rhs][t][z][y][x][4][3], device pointers, in the
 * given precision (OV_FP64: complex double, OV_FP32: complex float).  in and out must
 * not alias.  nrhs = 0 is a no-op.  Errors: INVALID_ARG, NO_GAUGE, OUT_OF_MEMORY, CUDA. */
int ov_apply_HW(ov_ctx* ctx, const void* in, void* out, int nrhs, int precision, void* stream);

/* Set an explicit quadrature: S_N = c0 + sum_j c_j (z_j - H)^-1, the weighted sum of
 * resolvents of Eqs. 5-7 (Eq. 7 gives the nodes z_j and weights rho w_j / N_q of one
 * ellipse; any list is accepted, e.g. a share of the nodes for a sharded sum).  z and c
 * point to n interleaved complex doubles on the host (copied); every Im z_j must be
 * nonzero.  n = 0 is allowed: then S_N = c0 (z and c may be NULL).
 * Errors: INVALID_ARG (n < 0, null arrays with n > 0, non-finite values, real node). */
int ov_set_contour(ov_ctx* ctx, int n, const double* z, const double* c, double c0_re, double c0_im);

/* Set the trapezoid rule of Eq. 7 on the ellipse z = gamma + rho (cos t + i alpha sin t),
 * theta_j = 2 pi (j - 1/2) / n_q.  OV_CONTOUR_SINGLE: c_j = 2 rho w_j / n_q, c0 = -1
 * (n_q nodes).  OV_CONTOUR_PAIR: c_j = +-rho w_j / n_q on the ellipses centred at
 * +-gamma, c0 = 0 (2 n_q nodes). */
int ov_set_contour_ellipse(ov_ctx* ctx, int n_q, double gamma, double rho, double alpha, int form);

/* Copy the current quadrature (the nodes and weights of Eqs. 5-7 set on the context) to
 * host arrays (z, c: room for *n complex doubles; on return *n is the node count).  Pass
 * z = c = NULL to query the count.  Errors: INVALID_ARG (n NULL, *n too small),
 * NO_CONTOUR. */
int ov_get_contour(const ov_ctx* ctx, int* n, double* z, double* c, double* c0);

/* Choose a single-contour ellipse of n_q nodes (Eq. 7; the paper tunes alpha, rho and
 * gamma by hand in "Numerical setup for the integration") from Lanczos bounds of H_W and
 * H_W^2 (`steps` Lanczos steps on each, from a fixed pseudo-random start) and set it on
 * the context.  The ellipse crosses the real axis at 0 and just beyond the upper
 * bound of the spectrum; alpha minimises the predicted method error.  `out` (may be
 * NULL) receives the bounds and the ellipse.  Work is enqueued on `stream` and waited
 * for.  Errors: INVALID_ARG (n_q < 2, steps < 4), NO_GAUGE, OUT_OF_MEMORY, CUDA. */
int ov_place_contour(ov_ctx* ctx, int n_q, int steps, ov_spectrum* out, void* stream);

/* Zolotarev node set (not in the paper, whose Summary leaves better quadrature rules to
 * future work): the optimal uniform rational approximation of sgn(lambda) on
 * [-lambda_max, -lambda_min] u [lambda_min, lambda_max] with n_poles pole pairs, written
 * as S = sum_j c_j (z_j - H)^-1 (c0 = 0) with 2 n_poles nodes z_j = +-i s_l on the
 * imaginary axis, ordered i s_1 .. i s_n, -i s_n .. -i s_1.  Built on the host from Jacobi
 * elliptic functions; *delta (may be NULL) receives the maximum error on the interval.
 * ov_zolotarev_rule needs no context or GPU: z, c receive 2 n_poles complex numbers
 * (interleaved re, im).  Errors: OV_ERR_INVALID_ARG unless 1 <= n_poles <= 128 and
 * 0 < lambda_min < lambda_max. */
int ov_zolotarev_rule(int n_poles, double lambda_min, double lambda_max, double* z, double* c, double* delta);
int ov_set_contour_zolotarev(ov_ctx* ctx, int n_poles, double lambda_min, double lambda_max, double* delta);

/* Spectral bounds as in ov_place_contour, then the Zolotarev node set on
 * [gap_lo, abs_max_bound]: gap_lo is the Lanczos estimate of min |lambda| lowered by the
 * residual bound of its H_W^2 Ritz value (by at most 20%).  out->gap = gap_lo,
 * out->predicted_error = delta, out->gamma = rho = alpha = 0. */
int ov_place_zolotarev(ov_ctx* ctx, int n_poles, int steps, ov_spectrum* out, void* stream);

/* out = S_N b ~= sgn(H_W) b for nrhs sources: sgn(H_W) = P_+ - P_- (Eq. 3), each
 * projector a contour integral of the resolvent (Eqs. 4, 5), the resolvents
 * y_j = (z_j - H_W)^-1 b (Eq. 6) of every node from one shifted Krylov solve, summed
 * with the quadrature weights of Eq. 7.  b, out: complex double, canonical layout
 * [rhs][t][z][y][x][4][3], device pointers (host pointers with opts->host_io); the
 * caller owns both; they must not alias.  stats may be NULL.
 * Errors: INVALID_ARG, NO_GAUGE, NO_CONTOUR, NOT_CONVERGED (out holds the last
 * iterate), BREAKDOWN (non-finite recurrence scalar, e.g. NaN in b), OUT_OF_MEMORY, CUDA. */
int ov_sgn_HW_apply(ov_ctx* ctx, const void* b, void* out, int nrhs, const ov_solve_opts* opts,
                    ov_stats* stats, void* stream);

/* out = D_ov(m_q) b = (1 + m_q)/2 b + (1 - m_q)/2 gamma5 S_N b (Eq. 1), S_N b as in
 * ov_sgn_HW_apply (same arguments, layouts, ownership and errors; m_q must be finite). */
int ov_overlap_apply(ov_ctx* ctx, double m_q, const void* b, void* out, int nrhs,
                     const ov_solve_opts* opts, ov_stats* stats, void* stream);

/* Gradients of L = Re <eta, S_N b> (one source), from the derivative of the resolvents
 * in Eq. 4, d(z - H)^-1 = (z - H)^-1 dH (z - H)^-1, with adjoint solves at conj(z_j):
 *   grad_b     = S_N^dag eta (complex double spinor): dL = Re <grad_b, db>;
 *   grad_links = dL/d omega_{x,mu,a} for U_mu(x) -> exp(i omega_a lambda_a/2) U_mu(x)
 *                (double [mu][t][z][y][x][8]).
 * Either output may be NULL.  Per-node forward y_j and adjoint (conj(z_j) - H)^-1 eta
 * solutions are kept in device memory during the call. */
int ov_sgn_vjp(ov_ctx* ctx, const void* eta, const void* b, void* grad_b, double* grad_links,
               const ov_solve_opts* opts, ov_stats* stats, void* stream);

/* Gradients of L = Re <eta, D_ov(m_q) b>: grad_b = (1+m_q)/2 eta + (1-m_q)/2 S_N^dag gamma5 eta,
 * grad_links = (1-m_q)/2 times the force of ov_sgn_vjp with eta -> gamma5 eta. */
int ov_overlap_vjp(ov_ctx* ctx, double m_q, const void* eta, const void* b, void* grad_b,
                   double* grad_links, const ov_solve_opts* opts, ov_stats* stats, void* stream);

/* Overlap solve: x = D_ov(m_q)^-1 b (Eq. 1 with the quadrature sign S_N of Eqs. 5-7), for
 * nrhs sources at once, by conjugate gradients on the normal equations
 * D^dag D x = D^dag b with D^dag = gamma5 D gamma5 (exact for the hermitian S_N).  Every
 * CG iteration applies D twice (each a full shifted solve with the options in `inner`;
 * NULL = defaults).  The products of iteration k are solved to the inner tolerance
 * inner->tol times max(1, ||r_0|| / (4 ||r_k||)) for the least converged source, at most
 * max(inner->tol, 1e-4): an error in a product matters in proportion to the current
 * residual, so later products need less accuracy (relaxed inexact Krylov); the true
 * residual below is checked with a product at inner->tol.  b, x: canonical complex128 spinors [nrhs][t][z][y][x][4][3], device
 * pointers (host pointers when inner->host_io), b != x; the caller owns both.  Stops a
 * source when ||D^dag (b - D x)|| <= tol ||D^dag b||; tol in (0, 1); at most max_iter
 * iterations.  stats: iterations = CG iterations, refine_rounds = D applies,
 * inner_iterations = Krylov iterations of all applies, max_residual = max over sources
 * of the true ||b - D x|| / ||b|| (one extra apply), error_bound = max normal-equation
 * residual.  Errors: OV_ERR_INVALID_ARG, OV_ERR_NO_GAUGE, OV_ERR_NO_CONTOUR,
 * OV_ERR_NOT_CONVERGED (x holds the last iterate; also when an inner solve misses its
 * tolerance), OV_ERR_BREAKDOWN, OV_ERR_OUT_OF_MEMORY, OV_ERR_CUDA.  A zero source gives x = 0. */
int ov_overlap_solve(ov_ctx* ctx, double m_q, const void* b, void* x, int nrhs, const ov_solve_opts* inner,
                     double tol, int max_iter, ov_stats* stats, void* stream);

/* FP32 stencil selection for ov_apply_HW(OV_FP32) (implementation choices of the H_W
 * stencil of Eq. 1; the paper has no counterpart).  Variants differ in layout, right-hand
 * sides per thread (link loads reused across them) and 12-real link compression (row 2
 * rebuilt as conj(row0 x row1)).  k = -1 (default): autotune -- each variant is timed
 * once on the live data per right-hand-side count and the fastest is kept.
 * ov_hw32_variants returns the number of variants and, for 0 <= k < count, describes
 * variant k.  Structure-of-arrays float2 layout: compressed 0 plain links, 1 12-real
 * links; rhs_tile = right-hand sides per thread, 0 = four threads per site (one per
 * direction, partial sums combined in shared memory).  compressed 8: spin-paired float4
 * layout (one 16-byte load per spin pair), one RHS per thread, 12-real links;
 * 9: right-hand-side-paired float4 layout (one float4 holds a component of two RHS,
 * paired FP32 instructions act on both) with compact 12-real links (48 B per link,
 * lanes broadcast in registers); 12: code 9 with row 2 rebuilt once in scalar
 * arithmetic (both lanes of a pair need the same value).  All read the diagonal term
 * before the hops, 128 threads per block except rhs_tile 0. */
int ov_set_hw32_variant(ov_ctx* ctx, int k);
int ov_hw32_variants(int k, int* rhs_tile, int* compressed, int* threads);

/* Launch structure of the Krylov loop (no counterpart in the paper).
 * enable = 1: the coefficient-space FP64 solve runs its whole iteration loop as one
 * cooperative persistent launch when the grid fits on the GPU (up to 16 sources);
 * enable = 0 (default): one launch per iteration phase, replayed from CUDA graphs
 * (measured faster on GB300 at 8^4: two grid barriers per iteration and L2-only
 * neighbour loads cost more than the launches and reduction tails they remove). */
int ov_set_persistent(ov_ctx* ctx, int enable);

/* Scheduling of independent sources (no counterpart in the paper).
 * Sources of one call are independent; the per-iteration kernels replayed from a CUDA
 * graph can run as `groups` parallel branches, each over a contiguous block of sources,
 * which fills the launch tails and serial reduction steps of small lattices and, on large
 * ones, runs one branch's vector update beside another's stencil.  groups = 0 (default):
 * one branch per source, at most four, when the stencil grid of all sources fits two
 * waves of the GPU, else two (six for the double-float mode); groups >= 1: that many
 * (capped at the source count of a batch).  Results do not depend on it (every source's
 * arithmetic is the same).
 * Errors: OV_ERR_INVALID_ARG for groups outside [0, 64]. */
int ov_set_concurrency(ov_ctx* ctx, int groups);

/* Kernel timing (instrumentation; no counterpart in the paper): when enabled, the library brackets every launch of its main
 * kernel classes with CUDA events on the launching stream and accumulates their
 * durations.  ov_kernel_times fills up to `cap` entries (name pointer, launches,
 * total ms) and returns the number of classes.  Disabled by default. */
int ov_set_kernel_timing(ov_ctx* ctx, int enable);
int ov_kernel_times(ov_ctx* ctx, const char** names, long long* launches, double* total_ms, int cap);

/* out = H_W in without allocating device memory (FP64, canonical layouts; U, in and
 * out are caller-owned device pointers on the current device; in != out).  The paper
 * has no counterpart: this serves callers that cannot call cudaMalloc -- a code that
 * hands all of HBM to its own pool up front, or a framework whose allocator must not
 * be bypassed (an allocation behind its back can fail, or take memory it has promised
 * elsewhere).  It needs no context.  Its staging buffers (structure-of-arrays copies
 * of U, in and out) live in one fixed 16 MiB device array inside the library, which
 * every GPU that loads the library holds until the process exits; a call needs
 * 576 V + 384 V nrhs bytes (V = sites, each part rounded up to 256 B) and larger
 * requests return OV_ERR_SCRATCH_TOO_SMALL.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress, with that device current) and
 * keeps it for the life of the process; do not use the entry point on a device after
 * cudaDeviceReset (the kept address belongs to the old context).  Every call on a device shares the one
 * array: calls that overlap on the GPU (different streams, or different host
 * threads) race and must be serialised by the caller.  Nothing in the array needs to
 * start at zero: each call writes all it reads.  Errors: INVALID_ARG (null or
 * aliasing pointers, nrhs < 1, dims < 1, |bc_t| != 1, m0 not finite),
 * SCRATCH_TOO_SMALL, CUDA (only for this call's own CUDA calls: an error the caller
 * left pending is neither cleared nor reported). */
int ov_apply_HW_noalloc(const int dims[4], int bc_t, double m0, const double* U, const void* in, void* out,
                        int nrhs, void* stream);

/* Library version string (no counterpart in the paper). */
const char* ov_version(void);

#ifdef __cplusplus
}
#endif

#endif /* OV_H_ */
