/*
 * pum.h -- C-ABI of the GB300 multilevel solver for partition-of-unity (PUM)
 * discretisations of the biharmonic and triharmonic equations, smoothed by the
 * fourth-kind Chebyshev iteration with block-FSAI preconditioners.
 *
 * Conventions used by every entry point
 * -------------------------------------
 *  - Block structure (Definition 2.1): a level with m x m patches has n = m*m
 *    block rows, uniform block size d = (p+1)(p+2)/2 (Section 5: dim V_i), and
 *    N = n*d unknowns.  Block row i = iy*m + ix; unknown (i, k) sits at i*d + k,
 *    k the local Legendre basis index ordered by total degree, then by the
 *    y-degree.
 *  - Levels are numbered 0 = finest ... n_levels-1 = coarsest.
 *  - Vector arguments are caller-owned DEVICE pointers to float64 arrays of the
 *    level's length N unless stated otherwise (typically torch tensors'
 *    data_ptr()).  The library never frees them.  All work is queued on the
 *    context's CUDA stream; calls return after queuing unless stated otherwise.
 *  - Every call returns a pum_status and never aborts.  On failure a message is
 *    available from pum_last_error().  Device-side conditions (non-positive
 *    Cholesky pivot, breakdown, a bounded wait on a shared-memory copy barrier
 *    that expired: PUM_ERR_TIMEOUT) are recorded in a device status word that
 *    the synchronous calls (bfsai_setup, pcg_solve, pum_sync) check before
 *    return.  No kernel traps or spins without a bound.
 *  - Threading: a context is used by one host thread at a time.
 */
#ifndef PUM_H
#define PUM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PUM_OK = 0,
  PUM_ERR_INVALID_ARG = 1, /* bad size, pointer, pattern or parameter           */
  PUM_ERR_OOM = 2,         /* device or host allocation failed                   */
  PUM_ERR_CUDA = 3,        /* a CUDA runtime call failed                         */
  PUM_ERR_NOT_SPD = 4,     /* non-positive pivot in a Cholesky factorisation     */
  PUM_ERR_BREAKDOWN = 5,   /* PCG: p^T A p <= 0 or a non-finite scalar           */
  PUM_ERR_NOCONV = 6,      /* PCG: maxit reached before rtol                     */
  PUM_ERR_TIMEOUT = 7,     /* a bounded device wait gave up                      */
  PUM_ERR_UNSUPPORTED = 8, /* a valid request this build does not implement      */
  PUM_ERR_IO = 9           /* file could not be read or written                  */
} pum_status;

typedef enum { PUM_F64 = 0, PUM_F32 = 1, PUM_BF16 = 2 } pum_dtype;

typedef struct pum_ctx pum_ctx;   /* device, stream, status word, last error    */
typedef struct pum_hier pum_hier; /* levels {A, P, P^T, G, G^T, beta}, coarse   */

/* A block-sparse (BSR) matrix with square d x d blocks stored row-major and
 * contiguous (block b occupies vals[b*bs*bs .. (b+1)*bs*bs)), columns sorted
 * within each block row.  Pointers are host memory unless on_device != 0. */
typedef struct {
  int32_t n_brows, n_bcols, bs;
  int64_t nnzb;
  const int32_t *row_ptr; /* n_brows + 1 */
  const int32_t *col_idx; /* nnzb        */
  const double *vals;     /* nnzb*bs*bs  */
  int32_t on_device;
} pum_bsr_view;

/* Host copy of a BSR matrix returned by pum_hier_export; free with pum_bsr_free. */
typedef struct {
  int32_t n_brows, n_bcols, bs;
  int64_t nnzb;
  int32_t *row_ptr;
  int32_t *col_idx;
  double *vals;
} pum_bsr_host;

/* The PUM problem of Section 4 / Examples 5.1 and 5.4 on the unit square. */
typedef struct {
  int32_t equation;     /* 4: Delta^2 u = f (Example 5.1); 6: -Delta^3 u = f (Example 5.4) */
  int32_t p;            /* local polynomial degree, 1..5                               */
  int32_t finest_m;     /* patches per side on the finest level (even while coarsening) */
  int32_t n_levels;     /* finest_m must be divisible by 2^(n_levels-1)               */
  double nitsche_c[3];  /* C_j of gamma^(j) = C_j (p+1)^2 h^-(order-1-2j); 0 -> default */
  int32_t quad_pts;     /* Gauss points per direction per sub-cell; 0 -> p + 6          */
  const double *f_coef; /* host, f_modes*f_modes coefficients c_ab (row a-1, column b-1) */
  int32_t f_modes;      /* f = sum c_ab (a^2+b^2)^(-f_decay/2) sin(a pi x) sin(b pi y)   */
  double f_decay;
  double aniso[3];      /* S11, S12, S22 of the SPD tensor S of Example 5.2 (equation 4 only):
                           S_ij S_kl u_,ijkl = f, Delta -> tr(S H), grad . n -> grad . (S n),
                           gamma^(0) scaled by |S|_2^2; all zero: isotropic (S = I)          */
} pum_problem;

enum { PUM_P0_LOWER = 0, PUM_P0_DIAG = 1 };

/* Block-FSAI set-up (Definition 2.2, Algorithm 1, Section 2.2). */
typedef struct {
  int32_t p0;       /* initial pattern: PUM_P0_LOWER = lower(P(A)), PUM_P0_DIAG = diagonal */
  int32_t adaptive; /* 0: static pattern P0; 1: Algorithm 1 from P0; 2: learned pattern
                       (the context's pattern model, pum_set_pattern_model) on levels of at
                       least 1024 block rows, each kept only when it passes the gate against
                       Algorithm 1 (pum_level_info.learned), Algorithm 1 elsewhere; not with
                       nested = 1 (PUM_ERR_INVALID_ARG)                                         */
  int32_t t_max;    /* adaptive steps (Algorithm 1)                                        */
  double tau;       /* threshold in (0, 1] (Algorithm 1)                                   */
  int32_t nested;   /* 1: one level of nesting (Section 2.2), same parameters twice        */
  double tie_rel;   /* argmin ties: smallest column with rho_c <= rho_min (1 + tie_rel)    */
} bfsai_params;

/* Smoother and cycle variants of Section 5 (the paper's comparisons). */
enum { PUM_SMOOTHER_CHEB4 = 0,      /* Algorithm 3, fourth-kind Chebyshev of degree k            */
       PUM_SMOOTHER_RICHARDSON = 1  /* k steps x <- x + M (b - A x): S = (I - M A)^k (Section 3.1) */
};
enum { PUM_CYCLE_VKK = 0,   /* V(k,k): the same smoother before and after (symmetric: CG)         */
       PUM_CYCLE_V2K0 = 1   /* V(2k,0): 2k steps before the coarse correction, none after
                               (non-symmetric: bicgstab_solve, not pcg_solve)                      */
};

/* Fourth-kind Chebyshev smoother (Algorithm 3) and its lambda_max estimate (Section 5). */
typedef struct {
  int32_t degree_k;      /* k >= 1 smoothing steps, pre and post (V(k,k))                  */
  int32_t lanczos_its;   /* Lanczos iterations (paper: 100)                                 */
  double lanczos_safety; /* beta = safety * lambda_max estimate (paper: 1.01)              */
  uint64_t lanczos_seed; /* SplitMix64 seed of the start vector; level l uses seed + l     */
  int32_t smooth_dt;     /* PUM_F64 or PUM_F32: storage and arithmetic of A, P and vectors  */
  int32_t g_dt;          /* PUM_F64, PUM_F32 or PUM_BF16 (BF16 needs smooth_dt = PUM_F32)   */
  int32_t mixed_levels;  /* FP32 form: the first mixed_levels levels keep their iterate and
                            right-hand side in FP64 (FP32 smoothing of corrections, residuals
                            with the FP64 operator, FP64 prolongation between such levels);
                            with mixed_levels > 0 the other levels post-smooth in correction
                            form with FP64-operator residuals; 0: plain FP32 cycle           */
  int32_t fp32_levels;   /* FP32 form: only the first fp32_levels levels store A, P, G and
                            vectors in FP32 (G in g_dt); the coarser ones smooth in FP64, for
                            Galerkin operators beyond FP32 (diagonal blocks with condition
                            numbers near 1/eps_32).  A level count below n_levels needs
                            fp32_levels <= mixed_levels (the switch happens under a mixed
                            level); >= n_levels: every level                                   */
  int32_t smoother;      /* PUM_SMOOTHER_CHEB4 or PUM_SMOOTHER_RICHARDSON                     */
  int32_t cycle;         /* PUM_CYCLE_VKK or PUM_CYCLE_V2K0                                   */
} smoother_params;

/* Outer preconditioned CG (one V(k,k) cycle as preconditioner). */
typedef struct {
  double rtol;        /* stop when ||r_j||_2 / ||b||_2 <= rtol (recursive residual)         */
  int32_t maxit;
  int32_t flexible;   /* 1: Polak-Ribiere beta (for a preconditioner in lower precision)    */
  double *hist;       /* host, maxit + 1 entries or NULL: ||r_j|| / ||b||, j = 0..iters    */
  int32_t iters;      /* out */
  int32_t converged;  /* out */
  double final_relres;/* out: last recursive residual                                       */
} pcg_report;

/* Per-level sizes and smoother data (for tests and reports). */
typedef struct {
  int32_t m, n, d;
  int64_t nnzb_A, nnzb_G, nnzb_GT, nnzb_P, nnzb_F0, nnzb_G1;
  double beta;        /* Chebyshev upper bound of this level (0 before bfsai_setup)        */
  double logdet_S;    /* sum_k log det S_kk of the (inner) FSAI (Lemma 2.7)                */
  int32_t coarsest;
  int32_t nested_inner; /* nested set-up: 1 inner FSAI of A1 = F0 A F0^T; 0 inner block Jacobi
                           (used when A1 is not numerically SPD in FP64; equals plain FSAI)  */
  int32_t fused_fsai;   /* 1: this level applies G^T G (nested: G1^T G1) reading G once --
                           partial products G_ji^T t_j, then a fixed-order gather (sliced FP32
                           levels; environment PUM_NO_FUSED_FSAI=1 at pum_create turns it off) */
  double flops_adapt;   /* FP64 flops (2 per multiply-add) of this level's Algorithm 1 kernel
                           at the last bfsai_setup, counted from the operations it performed  */
  double flops_factor;  /* FP64 flops of the FSAI factor kernel on the final patterns (from the
                           pattern sizes: Cholesky s^3/6, solves, S_kk, L_S and G = L_S^-1 F) */
  int32_t learned;      /* adaptive = 2: 1 when the level kept the learned pattern           */
  double gate;          /* adaptive = 2: the gate's shortfall (see pum_set_pattern_model); -1
                           when the level was not scored by the model                         */
  int32_t gg_rows, gg_parts, gg_ctas;  /* fused_fsai: the partial-product kernel's configuration
                           chosen at set-up by timing (block rows per group, consumer partitions
                           of a group's slots, persistent CTAs); 0 otherwise                  */
} pum_level_info;

/* Matrices selectable in pum_hier_export. */
enum { PUM_MAT_A = 0, PUM_MAT_P = 1, PUM_MAT_G = 2, PUM_MAT_GT = 3, PUM_MAT_F0 = 4, PUM_MAT_G1 = 5,
       PUM_MAT_A1 = 6 };

/* ---- context ------------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  Environment switches read here, each "1" to take
 * effect, for comparisons: PUM_NO_GRAPH (no CUDA graph of the V-cycle), PUM_NO_SELL (no sliced
 * layouts), PUM_NO_PDL (no programmatic dependent launch), PUM_NO_FUSED_FSAI (two-product FSAI
 * application), PUM_ADAPT_STEPS (Algorithm 1 with one launch per step and each row's local
 * systems factored from scratch, instead of one launch that carries every row through all its
 * steps with an incrementally grown factor).  cuda_stream is the cudaStream_t the library
 * queues all its work on (cudaStreamLegacy, i.e. (void*)1, selects the legacy default
 * stream); NULL makes the library create its own non-blocking stream, in which case the
 * caller must order its own use of the vectors with pum_sync.  Ownership of a passed
 * stream stays with the caller. */
pum_status pum_create(pum_ctx **ctx, int device, void *cuda_stream);
pum_status pum_destroy(pum_ctx *ctx);
/* Last error message of this context (never NULL; "" when none). */
const char *pum_last_error(const pum_ctx *ctx);
/* Wait for the context's stream and check the device status word. */
pum_status pum_sync(pum_ctx *ctx);

/* ---- hierarchy construction ---------------------------------------------------- */

/* Assemble the PUM problem (Section 4; Nitsche forms of Example 5.1 / 5.4) on the finest
 * level, build the L2-projection prolongations of Section 4 for every coarser level and
 * the Galerkin coarse operators A_{l-1} = P^T A_l P (Section 5), all on the device.
 * b_dev: device float64 array of length N_finest that receives the load vector l_n(.)
 * with zero boundary data (may be NULL).  *out is owned by the caller until
 * pum_hier_destroy.  Synchronous. */
pum_status pum_assemble(pum_ctx *ctx, const pum_problem *prob, pum_hier **out, double *b_dev);

/* Build a hierarchy from caller matrices (copied; caller keeps ownership).  A[0] is the
 * finest operator; for l >= 1, A[l] with vals == NULL is computed as P[l-1]^T A[l-1] P[l-1].
 * P[l] (l = 0..n_levels-2) maps level l+1 to level l (n_brows = n_l, n_bcols = n_{l+1}).
 * All blocks must share one block size: 3, 6, 10, 15 or 21 (the square's local spaces,
 * p = 1..5) or 20 (the cube's, p = 3: Example 5.3, whose matrices the caller assembles; the
 * library assembles the square only).  With 20 every level runs on the block-row kernels (no
 * sliced or fused layouts) and the learned pattern and multi-RHS products are not available.
 * Synchronous. */
pum_status pum_hier_from_bsr(pum_ctx *ctx, int n_levels, const pum_bsr_view *A, const pum_bsr_view *P,
                             pum_hier **out);

/* Block-FSAI smoothers for every level but the coarsest (static pattern, Algorithm 1, or
 * one level of nesting), the Lanczos estimate beta_l = safety * lambda_max(M_l A_l) per
 * level (Section 5), the explicit transposes used by the smoother, low-precision copies,
 * and the dense Cholesky factor of the coarsest operator.  Synchronous. */
pum_status bfsai_setup(pum_ctx *ctx, pum_hier *h, const bfsai_params *fp, const smoother_params *sp);

/* ---- hot path -------------------------------------------------------------------- */

/* Algorithm 3 on `level`: k steps of the M-preconditioned fourth-kind Chebyshev
 * iteration for A x = b, M = G^T G (or F0^T G1^T G1 F0 when nested).  x_is_zero != 0
 * means x0 = 0 (x is then output only).  b, x: device float64, length N_level; the
 * smoother runs in the set-up's smooth_dt. */
pum_status cheb4_smooth(pum_ctx *ctx, pum_hier *h, int level, const double *b, double *x, int x_is_zero);

/* z = B r for one V(k,k) cycle (Section 5): pre-smoothing from x0 = 0, residual,
 * restriction R = P^T, recursion, prolongation, post-smoothing with the same
 * polynomial; direct solve on the coarsest level.  r, z: device float64, N_finest. */
pum_status vcycle_apply(pum_ctx *ctx, pum_hier *h, const double *r, double *z);

/* Preconditioned CG from x = 0 for A_0 x = b (float64 throughout the outer iteration;
 * A_0 q products in float64).  b, x: device float64, N_finest.  Synchronous; fills rep.
 * Returns PUM_ERR_NOCONV when maxit is reached (x holds the last iterate). */
pum_status pcg_solve(pum_ctx *ctx, pum_hier *h, const double *b, double *x, pcg_report *rep);

/* BiCGStab (van der Vorst 1992) from x = 0 with one cycle as right preconditioner, the Krylov
 * method the Conclusions name for the non-symmetric V(2k,0) cycle (any cycle is accepted).
 * Shadow residual r^ = b.  float64 vectors and A_0 products; b, x: device float64, N_finest.
 * rep->hist gets ||r_j|| / ||b|| after each iteration (2 cycles and 2 products); rep->flexible
 * is ignored.  Synchronous; PUM_ERR_BREAKDOWN when r^.r, r^.v or t.t vanishes, PUM_ERR_NOCONV
 * at maxit (x holds the last iterate).  Work vectors are allocated on the first call. */
pum_status bicgstab_solve(pum_ctx *ctx, pum_hier *h, const double *b, double *x, pcg_report *rep);

/* Convergence factor rho_A of the stationary cycle (the measure of the paper's Section 5
 * figures): e_j = (I - B A) e_{j-1} for j = 1..n_cycles from the caller's e0 (device float64,
 * N_finest, not modified), rho = (e_n^T A e_n / e_0^T A e_0)^(1 / (2 n_cycles)).  *rho is a host
 * double.  Synchronous. */
pum_status pum_convergence_factor(pum_ctx *ctx, pum_hier *h, const double *e0, int n_cycles, double *rho);

/* ---- several right-hand sides of one problem ------------------------------------------ */

/* nrhs (1..16) right-hand sides at once: B and X are DEVICE float64 blocks, column c of length
 * N_finest at B + c N (X likewise, overwritten).  Every product of the V(k,k) cycle (Section 5,
 * Algorithm 3 smoothing) reads its matrix once for all columns (blocks of 4 or 16 columns, the
 * unused ones zero), and PCG runs for each column in lockstep from x0 = 0 with its own scalars,
 * stopping each column at ||r_c|| / ||b_c|| <= rtol (a finished column is left as it is).  The
 * cycle runs in the set-up's precision with FP64 outer PCG; in the FP32 form it is the plain FP32
 * cycle (every level's iterate and residual in FP32; mixed_levels is not used here), so every
 * smoothed level must be in one precision (fp32_levels >= n_levels - 1).  Non-nested FSAI and
 * V(k,k) only (PUM_ERR_UNSUPPORTED otherwise).  reps: nrhs reports; rtol, maxit and flexible are
 * read from reps[0], hist (if not NULL) from each.  PUM_ERR_NOCONV when a column did not reach
 * rtol.  Synchronous. */
pum_status pcg_solve_multi(pum_ctx *ctx, pum_hier *h, int32_t nrhs, const double *B, double *X, pcg_report *reps);
/* Z = the V(k,k) cycle applied to the nrhs columns of R (device float64 blocks as above). */
pum_status vcycle_apply_multi(pum_ctx *ctx, pum_hier *h, int32_t nrhs, const double *R, double *Z);

/* ---- batches of independent problems ---------------------------------------------------- */

/* bfsai_setup of n distinct hierarchies with the same parameters, by n_workers host threads,
 * thread w driving its own context workers[w] (distinct contexts on distinct streams).  status
 * (n entries, may be NULL)
 * receives each item's result; the return value is the first non-OK status in item order. */
pum_status pum_setup_batch(pum_ctx *const *workers, int n_workers, pum_hier *const *hs, int n,
                           const bfsai_params *fp, const smoother_params *sp, pum_status *status);

/* n solves on independent problems: item i solves hs[i] x[i] = b[i] (device float64 vectors of
 * that hierarchy's finest size) with pcg_solve (method 0) or bicgstab_solve (method 1), report
 * in reps[i] (hist, rtol, maxit, flexible as for the single solve).  Items of the same hierarchy
 * (several right-hand sides) run one after another on one worker; different hierarchies run
 * concurrently, one per worker thread and context.  Worker contexts must be distinct and run on
 * distinct streams (PUM_ERR_INVALID_ARG otherwise), and must not be used elsewhere during the
 * call.  status and the return value as for pum_setup_batch. */
pum_status pum_solve_batch(pum_ctx *const *workers, int n_workers, pum_hier *const *hs, int n,
                           const double *const *b, double *const *x, pcg_report *reps, int method,
                           pum_status *status);

/* pcg_solve_multi on n distinct hierarchies, concurrently as pum_solve_batch: item i solves the
 * nrhs columns of B[i] into X[i] (device blocks, column c at + c N_i), reports reps[i nrhs + c]
 * (rtol, maxit and flexible from reps[i nrhs]). */
pum_status pum_solve_batch_multi(pum_ctx *const *workers, int n_workers, pum_hier *const *hs, int n, int nrhs,
                                 const double *const *B, double *const *X, pcg_report *reps, pum_status *status);

/* ---- single steps of the hot path (device float64 vectors) ------------------------ */

/* r = b - A_level x (the residual of Algorithm 3). */
pum_status pum_residual(pum_ctx *ctx, pum_hier *h, int level, const double *b, const double *x, double *r);
/* z = M r, the block-FSAI application G^T (G r) (Definition 2.2) of the level. */
pum_status pum_fsai_apply(pum_ctx *ctx, pum_hier *h, int level, const double *r, double *z);
/* rc = P_level^T r: restriction from `level` to level+1 (Section 4). */
pum_status pum_restrict(pum_ctx *ctx, pum_hier *h, int level, const double *r, double *rc);
/* x += P_level e: prolongation from level+1 to `level`, added to x (Section 4). */
pum_status pum_prolong_add(pum_ctx *ctx, pum_hier *h, int level, const double *e, double *x);
/* z = A_c^{-1} r on the coarsest level (dense Cholesky). */
pum_status pum_coarse_solve(pum_ctx *ctx, pum_hier *h, const double *r, double *z);

/* ---- without allocation ------------------------------------------------------------- */

/* z = G^T (G r) for a caller-held block-FSAI factor G (square, block size 3/6/10/15/21) and
 * its explicit block transpose GT, both as DEVICE BSR arrays (on_device = 1, float64,
 * blocks contiguous d x d row-major, columns sorted; the pattern is not re-validated).
 * The paper has no counterpart.  It serves callers that cannot allocate device memory:
 * applications whose device memory is already reserved in full by another allocator (a
 * framework's caching pool), hosts with a fixed memory budget decided at start-up, and
 * latency-bound loops that cannot take the device-wide synchronisation cudaFree implies.
 * It calls no cudaMalloc/cudaFree and no allocating library routine: the intermediate G r
 * lives in a static device array of 2^20 doubles (8 MiB) that every GPU which loads the
 * library holds until the process exits, so G may have at most 1,048,576 unknowns (more:
 * PUM_ERR_INVALID_ARG with a message).  The first call on a device looks that array's
 * device address up (with the context's device made current for the call; the caller's
 * current device is restored before returning) and caches it, so make that first call
 * before any stream capture; a cudaDeviceReset of the device invalidates the cached
 * address for the rest of the process.  All calls share the array, and every call
 * overwrites the part it uses before reading it: calls whose work overlaps on the GPU
 * (other streams, or other contexts on the same device) race on it; calls queued on one
 * stream are ordered and safe.  r, z and the values: device float64, 8-byte aligned; r and
 * z of length n_brows*bs; the work is queued on the context's stream. */
pum_status pum_fsai_apply_noalloc(pum_ctx *ctx, const pum_bsr_view *G, const pum_bsr_view *GT, const double *r,
                                  double *z);

/* ---- learned candidate scoring for the adaptive pattern ------------------------------- */
/*
 * Not in the paper: an addition that shortens the set-up of Algorithm 1 (Section 2.1).  A
 * network scores the candidate blocks of every block row at once; each row takes its t_max
 * best-scoring candidates.  Candidates of row k: ring 1 = Algorithm 1's admissible set of P0_k
 * (c < k in the A-rows of P0_k, not in P0_k), ring 2 = the c < k in the A-rows of ring 1 in
 * neither.  The 12 features per (row, candidate) come from A and the static FSAI G0 on P0 (ring,
 * direct coupling |A_kc| / sqrt(|A_kk| |A_cc|), first-order gain g_c = |L_c^-1 (G0 A)_kc^T|_F^2
 * with A_cc = L_c L_c^T (Lemma 2.8's 1 - rho_c to first order), coupling through ring 1, the
 * rank and share of g_c in the row, the share of P0_k coupled to c, |P0_k|, the grid offset on
 * assembled hierarchies, the row's fill and its ring-1 size), as float32.
 * The network: 12 -> 64 -> 64 -> 1 with ReLU; the products use BF16 weights (round to nearest
 * even of the FP32 master weights) with FP32 accumulation; biases FP32.  Training minimises the
 * mean binary cross-entropy of the logit against the label "Algorithm 1 chose this candidate"
 * with Adam (Kingma and Ba 2015) on the device.
 * The gate (adaptive = 2): on every 16th block row of a level, Algorithm 1 runs as well; with
 * L the sum of log det S_kk over those rows (Lemma 2.7's measure up to a constant) for the
 * learned pattern, A1 for Algorithm 1's and P for P0, the shortfall (L - A1) / (P - A1) must be
 * at most 0.05 (the learned pattern reaches 95% of Algorithm 1's gain), else the level runs
 * Algorithm 1 on every row.
 */
#define PUM_MLP_FEATURES 12
#define PUM_MLP_HIDDEN 64
/* Parameters (FP32 master copy), row-major: w1[o][f], w2[o][i]. */
typedef struct {
  float w1[PUM_MLP_HIDDEN * PUM_MLP_FEATURES];
  float b1[PUM_MLP_HIDDEN];
  float w2[PUM_MLP_HIDDEN * PUM_MLP_HIDDEN];
  float b2[PUM_MLP_HIDDEN];
  float w3[PUM_MLP_HIDDEN];
  float b3;
} pum_mlp;

/* Candidates of one level (library-owned DEVICE arrays, free with pum_candidates_free):
 * n candidates, rows ascending, ring 1 then ring 2 within a row (each ascending). */
typedef struct {
  int64_t n;
  int32_t *row, *col;  /* block row and candidate column                                   */
  float *x;            /* n x PUM_MLP_FEATURES, row-major                                    */
  float *y;            /* label: 1 when the level's current FSAI pattern holds the candidate */
} pum_candidates;

/* Candidates, features and labels of a set-up level (non-nested): the pools and features are
 * those of the hierarchy's P0 (bfsai_params.p0 of the last bfsai_setup), the labels those of
 * its current pattern (Algorithm 1's after an adaptive set-up).  Synchronous. */
pum_status pum_fsai_candidates(pum_ctx *ctx, pum_hier *h, int level, pum_candidates *out);
void pum_candidates_free(pum_candidates *c);
/* Copy the candidate arrays into caller DEVICE buffers (any may be NULL; row/col n entries,
 * x n*PUM_MLP_FEATURES, y n), on the context's stream. */
pum_status pum_candidates_copy(pum_ctx *ctx, const pum_candidates *c, int32_t *row, int32_t *col, float *x, float *y);
/* logits[i] of the features x[i] (device float32 arrays, n rows). */
pum_status pum_mlp_forward(pum_ctx *ctx, const pum_mlp *m, const float *x, int64_t n, float *logits);
/* Mean binary cross-entropy of the logits of x against y (device float32, n rows) and its
 * gradient with respect to every parameter (host outputs; the BF16 rounding is passed through
 * as the identity).  Deterministic (fixed-order reductions).  Synchronous. */
pum_status pum_mlp_grad(pum_ctx *ctx, const pum_mlp *m, const float *x, const float *y, int64_t n, double *loss,
                        pum_mlp *grad);
/* Adam on the device from the parameters in *m (updated in place on return): `epochs` passes
 * over the n samples in a seeded random order (SplitMix64), minibatches of `batch`, step size
 * lr, beta1 0.9, beta2 0.999, eps 1e-8.  loss (may be NULL): mean loss over all n samples
 * after training.  Synchronous. */
pum_status pum_mlp_train(pum_ctx *ctx, pum_mlp *m, const float *x, const float *y, int64_t n, int32_t epochs,
                         int32_t batch, double lr, uint64_t seed, double *loss);
/* The model bfsai_setup uses with adaptive = 2 (copied; NULL removes it). */
pum_status pum_set_pattern_model(pum_ctx *ctx, const pum_mlp *m);

/* ---- inspection, persistence ------------------------------------------------------- */

pum_status pum_hier_levels(const pum_hier *h, int *n_levels);
pum_status pum_level_info_get(const pum_hier *h, int level, pum_level_info *info);
/* Host copy of a level's matrix (float64 values); free with pum_bsr_free.  Synchronous. */
pum_status pum_hier_export(pum_ctx *ctx, const pum_hier *h, int level, int which, pum_bsr_host *out);
void pum_bsr_free(pum_bsr_host *m);
/* Versioned binary file of the whole set-up product (all levels' matrices, betas,
 * coarse factor, parameters).  load rebuilds a hierarchy ready for the hot path. */
pum_status pum_hier_save(pum_ctx *ctx, const pum_hier *h, const char *path);
pum_status pum_hier_load(pum_ctx *ctx, const char *path, pum_hier **out);
pum_status pum_hier_destroy(pum_hier *h);

/* ---- measurement -------------------------------------------------------------------- */

/* Per-kernel-class timing of the hot path.  When enabled, every launch of the classes
 * below on the finest level is bracketed by CUDA events recorded on the launching
 * stream (inside the captured V-cycle graph when one is used); pum_timing_read returns,
 * per class, the number of launches and the summed event time since the last reset.
 * Class ids: 0 residual b - A x in the smoother's precision, 1 G r, 2 G^T t + Chebyshev
 * update, 3 A p in PCG, 4 residual with the FP64 operator on FP32 vectors; set-up classes
 * (every level): 5 the Algorithm 1 kernel (all steps of all rows), 6 the FSAI factor
 * kernel (G on the final patterns). */
enum { PUM_TK_RESID = 0, PUM_TK_G = 1, PUM_TK_GT = 2, PUM_TK_PCG_AP = 3, PUM_TK_RESID64 = 4, PUM_TK_ADAPT = 5,
       PUM_TK_FACTOR = 6, PUM_TK_COUNT = 7 };
#define PUM_TIMING_ALL ((1 << PUM_TK_COUNT) - 1)
/* mask: bit k times class k (PUM_TIMING_ALL: every class; 0: off).  Timing only the classes
 * of interest keeps the other launches free of event records. */
pum_status pum_timing_enable(pum_ctx *ctx, int mask);
pum_status pum_timing_reset(pum_ctx *ctx);
pum_status pum_timing_read(pum_ctx *ctx, int64_t *launches, double *ms);
/* Number of kernels of this library launched on the context since creation. */
int64_t pum_launch_count(const pum_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* PUM_H */
