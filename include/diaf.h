/*
 * diaf.h -- C ABI of the GB300 library for the columnwise construction of
 * sparse W, V with AW ~ V ("direct approximate factoring of the inverse",
 * Byckling & Huhtanen), and for applying the resulting right preconditioner
 * A^-1 ~ W V^-1 (eq. afac, Sec. 2).
 *
 * Conventions for every entry point:
 *  - Sparse matrices and patterns are CSC, 0-based, int32 indices, the row
 *    indices of each column strictly increasing.  n and every nnz < 2^31.
 *  - Pointers named d_* (and every pointer inside diaf_csc / diaf_pattern /
 *    diaf_vspec) are DEVICE pointers on the current CUDA device; h_* are host
 *    pointers.  Inputs stay owned by the caller and must remain valid until
 *    the work enqueued on `stream` has finished.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *    Calls enqueue their work on it in order.  Calls that must size their
 *    outputs from the data (diaf_factor, the first diaf_apply) synchronise
 *    `stream`, as noted.
 *  - Complex values are interleaved (re, im) doubles (DIAF_C128).
 *  - Every function returns diaf_status; nothing throws across the ABI.
 *    After a non-OK status, diaf_last_error() gives a one-line reason
 *    (thread-local, valid until the next call on the same thread).
 *  - A missing or non-sm_103 device gives DIAF_ECUDA; there is no CPU path.
 */
#ifndef DIAF_H
#define DIAF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DIAF_OK = 0,
  DIAF_EINVAL = 1,       /* bad argument: null pointer, size, unsorted / out-of-range index */
  DIAF_ENOMEM = 2,       /* device allocation failed */
  DIAF_ECUDA = 3,        /* CUDA runtime error (no device, launch failure, ...) */
  DIAF_ENUMERIC = 4,     /* non-finite values produced */
  DIAF_ETIMEOUT = 5,     /* a bounded device-side wait ran out (no current call waits on the device) */
  DIAF_EUNSUPPORTED = 6  /* a column's tile exceeds every compiled kernel's capacity */
} diaf_status;

/* Value type of A (and therefore of W and V). */
enum { DIAF_F64 = 0, DIAF_C128 = 1 };

/* The two basic algorithms.  DIAF_ALG_Q: columns of V of unit norm, v_j from
 * eq. nocond, w_j from the least-squares problem eq. condwj (Sec. 2.1, the
 * "first basic algorithm", DIAF-Q).  DIAF_ALG_S: columns of W of unit norm,
 * w_j the right singular vector of the smallest singular value of A_j with
 * the rows I_j removed, v_j = P_V A w_j (Sec. 2.2, the "second basic
 * algorithm", DIAF-S). */
enum { DIAF_ALG_Q = 1, DIAF_ALG_S = 2 };

/* Arithmetic of the numeric phase.  DIAF_PREC_FP64: everything in FP64
 * (complex128 for DIAF_C128).  DIAF_PREC_MIXED32: QR, leverage keys and
 * Jacobi in FP32 (complex64) on an FP64 tile, then an FP64 refinement of
 * (w_j, v_j) against the FP64 tile and an FP64 residual.  A column whose FP32
 * leverage decision lies within the FP32 error bound of its threshold gets
 * its leverage keys recomputed in FP64 (the FP64 path's own QR and key
 * routines), so I_j is the FP64 choice; a column whose tile is too
 * ill-conditioned for FP32 factors, or whose refinement cannot converge, is
 * computed by the FP64 path instead (flag DIAF_FLAG_FP64_FALLBACK). */
enum { DIAF_PREC_FP64 = 0, DIAF_PREC_MIXED32 = 1 };

/* How I_j (the pattern of column j of V) is obtained.  FIXED: given pattern.
 * UPPER / LOWER / ALL: the optimal-V rule of Sec. 3.1 -- the diagonal j plus
 * the l_j - 1 admissible rows of the tile with the largest leverage
 * h_i = ||Q_j(i,:)||^2 (the columns of Q_j^* of largest norm).  Admissible
 * rows: i < j (UPPER, V upper triangular as in the Gauss-Seidel structure of
 * Sec. 4.2), i > j (LOWER), any i != j (ALL); always rows of the tile. */
enum { DIAF_RULE_FIXED = 0, DIAF_RULE_UPPER = 1, DIAF_RULE_LOWER = 2, DIAF_RULE_ALL = 3, DIAF_RULE_BLOCK = 4 };

/* Per-column flag bits (col_flags). */
enum {
  DIAF_FLAG_RANK_DEFICIENT = 1,  /* S: sigma_min <= 1e-14 sigma_max or fewer tile rows than k_j outside I_j;
                                    Q: a pivot of R below 1e-14 max|R_ii| (its w entry set to 0) */
  DIAF_FLAG_DEGENERATE = 2,      /* the optimal vector is not unique to 1e-6 relative gap
                                    (S: smallest two singular values, Q: largest two) */
  DIAF_FLAG_VJJ_ZERO = 4,        /* |v_jj| <= 64 eps ||v_j|| (V singular at j to rounding); phase taken from w */
  DIAF_FLAG_JACOBI_NOCONV = 8,   /* the Jacobi SVD hit its 30-sweep limit */
  DIAF_FLAG_NONFINITE = 16,      /* NaN or Inf in w_j, v_j or res_j */
  DIAF_FLAG_EMPTY = 32,          /* k_j = 0 (empty W column) */
  DIAF_FLAG_FP64_FALLBACK = 64,  /* mixed precision: the column was computed by the FP64 path (a tile
                                    too ill-conditioned for FP32 factors, a refinement that cannot
                                    converge, or a large tile of complex A or DIAF-Q) */
  DIAF_FLAG_STABILISED = 128     /* DIAF-Q: v_jj was imposed (stabilised column of Sec. 3.2) */
};

typedef struct {
  int32_t n;
  int64_t nnz;
  const int32_t* colptr; /* device, n+1 */
  const int32_t* rowidx; /* device, nnz */
  const void* vals;      /* device, nnz doubles (F64) or 2*nnz doubles (C128) */
  int32_t dtype;         /* DIAF_F64 or DIAF_C128 */
} diaf_csc;

typedef struct {
  int32_t n;
  int64_t nnz;
  const int32_t* colptr; /* device, n+1 */
  const int32_t* rowidx; /* device, nnz */
} diaf_pattern;

typedef struct {
  int32_t rule;               /* DIAF_RULE_* */
  const diaf_pattern* fixed;  /* rule == FIXED: the V pattern; else ignored */
  const int32_t* budget;      /* device int32[n]: l_j including the diagonal (values < 1 act as 1),
                                 capped by 1 + the number of admissible rows; NULL = all admissible */
  double tie_tol;             /* leverage keys within tie_tol of the current largest count as tied and the
                                 lower row is taken; <= 0 selects the default 1e-9 */
  /* Stabilised DIAF-Q (Sec. 3.2; ignored by DIAF-S): where the unit v_j of
   * eq. nocond has |v_jj| < stab_tol, v_jj is imposed as stab_r (<= 0: 2, the
   * value of the paper's experiments) and the other entries are the top
   * singular vector of Q(I_j without j, :)^* with the phase that maximises
   * ||Q(I_j,:)^* v_j||; v_j is then scaled to unit norm and w_j solves
   * eq. condwj as before (flag DIAF_FLAG_STABILISED).  stab_tol <= 0 turns it
   * off; the paper's experiments use 1e-2.  Zero-initialised structs keep
   * the plain method. */
  double stab_tol;
  double stab_r;
  /* DIAF_RULE_BLOCK (block-diagonal V, Sec. 5's experiments): device int32[n],
   * the block of every row, non-decreasing in row order (so every block is a
   * contiguous range of rows); the admissible rows of column j are the other
   * rows of j's block.  diaf_apply then factors each diagonal block of V by
   * dense LU with partial pivoting (blocks of at most 64 rows; larger ones make
   * diaf_apply return DIAF_EUNSUPPORTED).  Copied at factorisation. */
  const int32_t* blocks;
} diaf_vspec;

typedef struct diaf_factors diaf_factors; /* opaque, library-owned */

/*
 * diaf_factor -- the whole setup: for every column j, gather the tile
 * T = A(R_j, J_j) of the rows R_j touched by the columns J_j of the W
 * pattern (A_j of eq. spaqr on its nonzero rows), QR it (eq. spaqr), choose
 * I_j (Sec. 3.1 rule or fixed), solve DIAF-S (Sec. 2.2) or DIAF-Q (Sec. 2.1)
 * for (w_j, v_j), fix the phase so that v_jj is real and >= 0 (allowed by the
 * scaling-invariance theorem of Sec. 2.1), and scatter into CSC W (pattern
 * PW) and V (pattern I_j).  res_j = ||A w_j - v_j||_2 per column.
 *   A       : the n x n matrix (values F64 or C128).
 *   PW      : W pattern (J_j = column j), PW->n == A->n.
 *   V       : V pattern specification.
 *   alg     : DIAF_ALG_Q or DIAF_ALG_S.   prec: DIAF_PREC_*.
 *   out     : receives a new handle; free with diaf_free.
 * Synchronises `stream` twice (in the symbolic pass: to size the row-union
 * storage, then V and the size buckets).  The
 * numeric work is enqueued on `stream`; the outputs are ready when it has
 * run.  Errors: EINVAL (arguments, unsorted / out-of-range indices),
 * ENOMEM, ECUDA, EUNSUPPORTED (a column needs more than 4096 gathered
 * entries or a tile beyond 1024 x 64).
 */
diaf_status diaf_factor(const diaf_csc* A, const diaf_pattern* PW, const diaf_vspec* V, int32_t alg,
                        int32_t prec, void* stream, diaf_factors** out);

/* Launch tuning of the numeric pass (diaf_factor_tuned, diaf_plan_create,
 * found by diaf_autotune).  Zero fields select the defaults.
 *   m_edge0: tiles with max(m_j, k_j) <= m_edge0 (and k_j <= 16) run in size
 *            bucket 0 (warp per column, 32-row tile); 1..32, default 32.
 *   m_edge1: tiles up to m_edge1 rows (k_j <= 32) run in bucket 1 (warp per
 *            column, 64-row tile); 1..64, default 64.  Larger tiles run in
 *            bucket 2 (one 256-thread CTA per column).
 *   warps_per_block[b]: CTA size of the warp kernels of buckets 0 and 1
 *            (1..8; 0 = the most warps resident per SM).
 *   small_tiles: bucket 0 of real DIAF-S in mixed precision: 0 (default) or
 *            1 = four lanes per column (a warp runs eight columns; columns it
 *            cannot finish in FP32 go on to the warp kernel), 2 = one warp
 *            per column.
 *   large_tiles: bucket 2 of real DIAF-S in mixed precision: 0 (default) or
 *            1 = the tensor-core Gram path (G = T^T T on the tensor cores,
 *            Cholesky factors, for column-scaled kappa <= 30; other tiles
 *            keep the Householder QRs), 2 = Householder QRs only. */
typedef struct {
  int32_t m_edge0;
  int32_t m_edge1;
  int32_t warps_per_block[2];
  int32_t small_tiles;
  int32_t large_tiles;
} diaf_tuning;

typedef struct {
  int32_t n;
  int32_t dtype;
  int32_t alg;
  int32_t prec;
  int64_t nnz_w;       /* = nnz(PW) */
  int64_t nnz_v;       /* = sum_j l_j */
  int32_t max_k, max_m, max_l;
  int32_t n_buckets;   /* number of size buckets launched */
  int32_t bucket_cols[8];
} diaf_factor_info;

/* Sizes and bucket statistics of a factorisation (host copy; no sync):
 * bookkeeping of the column-wise setup of Sec. 2, no passage of its own.
 * Errors: EINVAL (NULL F or info). */
diaf_status diaf_factor_info_get(const diaf_factors* F, diaf_factor_info* info);

/* diaf_factor (Sec. 2.1, 2.2, 3.1) with launch tuning (NULL = defaults);
 * the tuning changes only how the independent columns are batched, never a
 * result.  Arguments, ownership and errors as diaf_factor, plus EINVAL for
 * tuning values out of range. */
diaf_status diaf_factor_tuned(const diaf_csc* A, const diaf_pattern* PW, const diaf_vspec* V, int32_t alg,
                              int32_t prec, const diaf_tuning* tuning, void* stream, diaf_factors** out);

/* Times the numeric pass of diaf_factor_tuned over the bucket edges and the
 * warp kernels' CTA sizes (coordinate descent, best of two runs per point)
 * and returns the fastest tuning (*best, host) and its numeric-pass time in
 * ms (*best_ms, host).  Runs about 15 factorisations of the given problem.
 * Launch tuning of the column-parallel setup (Sec. 2), not a passage of the
 * paper.  Errors as diaf_factor. */
diaf_status diaf_autotune(const diaf_csc* A, const diaf_pattern* PW, const diaf_vspec* V, int32_t alg, int32_t prec,
                          void* stream, diaf_tuning* best, float* best_ms);

/* A factorisation plan: the symbolic pass done once, the numeric pass
 * (gather, QR, V rule, DIAF solve, scatter -- every size bucket) captured in
 * one CUDA graph.  For repeated factorisations of matrices with the same
 * structure (new values written into the same A->vals buffer, e.g. a
 * time-stepping operator), diaf_plan_execute replays the graph: one launch,
 * no host synchronisation, no allocation.  The plan keeps A's, PW's and the
 * V specification's device arrays by pointer: they must stay valid and
 * unchanged except A's values.  diaf_plan_create synchronises `stream`; it
 * does not run the numeric pass. */
typedef struct diaf_plan diaf_plan;
/* Errors of diaf_plan_create as diaf_factor (*out receives the plan; free
 * with diaf_plan_free). */
diaf_status diaf_plan_create(const diaf_csc* A, const diaf_pattern* PW, const diaf_vspec* V, int32_t alg,
                             int32_t prec, const diaf_tuning* tuning, void* stream, diaf_plan** out);
/* Enqueues the numeric pass on `stream` (one graph launch); the plan's
 * factors are ready when it has run.  Executions must not overlap.
 * Errors: EINVAL (NULL plan), ECUDA (graph launch). */
diaf_status diaf_plan_execute(diaf_plan* P, void* stream);
/* The plan's factors (borrowed; freed by diaf_plan_free; NULL for NULL). */
diaf_factors* diaf_plan_factors(diaf_plan* P);
/* Frees the plan, its graph and its factors.  NULL is ignored. */
void diaf_plan_free(diaf_plan* P);

/* Timings of a factorisation from CUDA events recorded on its stream (waits
 * for them): ms[0] the whole diaf_factor call (first to last enqueued work,
 * host synchronisations included), ms[1] the numeric pass, ms[2 + b] the
 * numeric kernel of size bucket b (0 when the bucket was empty).  nms is the
 * capacity of ms (host floats) and must be >= 2 + n_buckets.  Measurement,
 * not a passage of the paper.  Errors: EINVAL (NULL, nms too small), ECUDA. */
diaf_status diaf_factor_timings(const diaf_factors* F, float* ms, int32_t nms);

/* Mixed precision: the number of columns per size bucket that the FP64 path
 * computed (flag DIAF_FLAG_FP64_FALLBACK; in the large-tile bucket every
 * column for complex A or DIAF-Q, the handed-back ones for real DIAF-S);
 * zeros for the FP64 form.  Waits for F's stream.  nb >= n_buckets. */
diaf_status diaf_factor_fallbacks(const diaf_factors* F, int32_t* counts, int32_t nb);

/* Number of CUDA kernels this library has launched in this process
 * (instrumentation; never fails). */
long long diaf_launch_count(void);

/* Numbers of apply preparations (first diaf_apply calls on triangular V) in
 * this process that built the level schedule from V's structure as it
 * reached the host during the numeric pass (`streamed`: factors of rules
 * UPPER / LOWER made by diaf_factor or diaf_factor_tuned while no other such
 * factorisation held the library's one host-mapped copy of V's structure),
 * and that copied V's structure to the host after the numeric pass
 * (`copied`: every other case).  Either pointer may be NULL.
 * (Instrumentation, no passage of the paper; never fails.) */
void diaf_apply_prep_counts(int64_t* streamed, int64_t* copied);

/* Caps the device memory that the setup and apply paths (diaf_factor,
 * diaf_factor_tuned, diaf_plan_*, diaf_apply and the factor handles they
 * keep) may hold at one time, over all handles of the process: bytes > 0 is
 * the cap, 0 removes it (the default).  An allocation that would exceed the
 * cap is not attempted: the call that needed it frees what it had taken and
 * returns DIAF_ENOMEM.  Lowering the cap below the bytes already held frees
 * nothing; only later allocations are refused.  (Resource control, no passage
 * of the paper; the Krylov solvers, the learned proposal and the sparsified
 * powers are not counted.)  Errors: EINVAL (bytes < 0). */
diaf_status diaf_set_device_memory_limit(int64_t bytes);

/* Device bytes the setup and apply paths hold now (what the cap above
 * counts).  Never fails. */
int64_t diaf_device_memory_in_use(void);

/* The setup and apply paths allocate from a stream-ordered memory pool of
 * the library's own (one per device) that keeps what they free, so that the
 * next setup reuses it without mapping new pages; the pool therefore holds
 * the high-water mark of the library's use.  This call returns the pool's
 * unused memory on the current device to the driver (memory still held by
 * live handles stays).  Call it with no setup or apply of the library in
 * flight on that device.  (Resource control, no passage of the paper.)
 * Errors: ECUDA. */
diaf_status diaf_release_pool_memory(void);

/* Borrowed device views of the outputs (valid until diaf_free): the W and V
 * of eq. afac (Sec. 2.3), column j of each from Sec. 2.1 / 2.2, and
 * res_j = ||A w_j - v_j||.  W: colptr/rowidx = copies of PW, vals nnz_w
 * scalars;  V: CSC with column j on I_j (sorted), vals nnz_v scalars;
 * col_res: double[n];  col_flags: uint32[n] (DIAF_FLAG_* bits).  Any output
 * pointer may be NULL.  Errors: EINVAL (NULL F). */
diaf_status diaf_get_factors(const diaf_factors* F, diaf_csc* W, diaf_csc* V, const double** col_res,
                             const uint32_t** col_flags);

/* y = W V^-1 x (eq. afac: A^-1 ~ W V^-1, right preconditioning, Sec. 2.3).
 * x, y: device vectors of n scalars (dtype of F), must not overlap.  V must
 * be triangular (rules UPPER / LOWER, or a fixed triangular pattern) with a
 * nonzero diagonal.  The first call on F prepares the apply: row-oriented
 * copies of W and V and the level schedule of the V solve (the depth of each
 * row in V's dependency graph, computed on the host; this first call
 * allocates, and waits on the host for the preparation's work on `stream`
 * (the numeric pass included); it returns while its solve may still run --
 * make it before any stream capture).  The level-ordered V holds each row
 * scaled by 1/diag, and W's row-oriented copy is built on a side stream of
 * the library while the solve runs (the SpMV waits for it).
 * For factors of rules UPPER / LOWER made by diaf_factor(_tuned), the column
 * kernels also write V's row indices into a host-mapped buffer of the
 * library as each column is finished (the columns of an upper V in
 * descending order), and this first call builds the schedule from the
 * columns as they arrive, while the numeric pass still runs.  One
 * factorisation at a time holds that buffer, from diaf_factor until its
 * first diaf_apply or diaf_free; the others copy V's structure after the
 * numeric pass (same schedule, later).
 * Later calls only enqueue three kernels: the scaling of x by 1/diag (all
 * SMs), the level-scheduled triangular solve (one block, a barrier between
 * levels) and the W SpMV.  Errors: EINVAL (V not triangular or zero
 * diagonal -- found by the first call, whose y is then not valid), ENOMEM,
 * ECUDA. */
diaf_status diaf_apply(diaf_factors* F, const void* x, void* y, void* stream);

/* The level schedule of the apply's triangular solve, on the host (no GPU
 * call): V given by its columns in host arrays (colptr int32[n+1] with
 * colptr[0] = 0, rowidx int32[colptr[n]], rows in any order within a
 * column; the values are not looked at).  level[i] (host int32[n], written)
 * receives the depth of row i in V's dependency graph -- row i waits for t_j
 * when V(i,j) != 0, i != j, so rows of one level are independent (the
 * level-scheduled form of the substitution in eq. afac's V^-1, Sec. 2.3);
 * *nlev the number of levels (max level + 1, 0 when n = 0); *upper 1 for an
 * upper (or diagonal) V, 0 for a lower one.  This is the pass diaf_apply
 * runs when it prepares the solve.  Errors: EINVAL -- NULL pointer, n < 0,
 * malformed colptr, a row index out of range, V neither upper nor lower
 * triangular, or a missing diagonal entry. */
diaf_status diaf_level_schedule(int32_t n, const int32_t* colptr, const int32_t* rowidx, int32_t* level,
                                int32_t* nlev, int32_t* upper);

/* y = W V^-1 x exactly as diaf_apply computes it, but allocating nothing.
 * (The paper has no counterpart: this is an interface for callers that must
 * not allocate device memory when they apply the preconditioner -- code
 * running inside a device-memory budget fixed at start-up, or a host
 * framework whose allocator owns all device memory and forbids allocations
 * by the libraries it calls.)
 * Such callers set up beforehand: diaf_factor, then one diaf_apply on F,
 * which builds the row-oriented copies of W and V.  Without that first
 * diaf_apply this call returns DIAF_EINVAL.
 * Its one piece of scratch, t = V^-1 x, is a fixed device array of 4 MB
 * inside the library, held by every GPU that loads it until the process
 * exits; n is limited to 262,144 rows (DIAF_EINVAL beyond).  The solve is
 * diaf_apply's level-scheduled one and writes all of t before reading it, so
 * nothing has to be cleared between calls.  The first call on each device
 * looks up the array's device address (cached for the process: do not use
 * this entry point across a cudaDeviceReset); make that first call before
 * any stream capture.  All calls on a device share the array, so calls that
 * overlap on the GPU (different streams, or several host threads) race:
 * serialise them.  x, y as for diaf_apply. */
diaf_status diaf_apply_static(diaf_factors* F, const void* x, void* y, void* stream);
/* (Triangular V only: factors of DIAF_RULE_BLOCK give DIAF_EUNSUPPORTED.) */

/* Waits for `stream` and reports device-side errors recorded by earlier
 * calls on F (capacity overflows) as a status (infrastructure, no passage of
 * the paper).  Errors: EINVAL (NULL F), EUNSUPPORTED as recorded, ECUDA. */
diaf_status diaf_sync(diaf_factors* F, void* stream);

/* Frees F and every device buffer it owns (stream-ordered on the stream F was
 * created on; that stream must still exist).  When F still holds the host
 * copy of V's structure (no diaf_apply was made on it), it first waits for
 * that stream.  NULL is ignored.  Never fails. */
void diaf_free(diaf_factors* F);

typedef struct diaf_solver diaf_solver; /* opaque: A in row-oriented form for Krylov solves */

/* Prepares A for the Krylov solvers of Sec. 5 (row-oriented copy of the
 * caller's CSC, owned by the solver; allocates).  Errors: EINVAL (NULL, bad
 * sizes), ENOMEM, ECUDA. */
diaf_status diaf_solver_create(const diaf_csc* A, void* stream, diaf_solver** out);
/* Frees the solver.  NULL is ignored. */
void diaf_solver_free(diaf_solver* S);

typedef struct {
  int32_t iterations;   /* iterations performed */
  int32_t converged;    /* 1 when ||r|| <= tol ||r0|| */
  int32_t breakdown;    /* 1 on a zero denominator (the paper's double dagger) */
  double relres;        /* final ||r|| / ||r0|| */
} diaf_solve_info;

/* Right-preconditioned BiCGSTAB on A x = b (Sec. 5: x0 = 0, stop when the
 * residual is reduced by tol, at most maxit iterations).  F == NULL solves
 * without preconditioner.  b, x: device vectors of n scalars.  One
 * device-to-host read per iteration (the convergence test). */
diaf_status diaf_bicgstab(diaf_solver* S, diaf_factors* F, const void* b, void* x, double tol, int32_t maxit,
                          void* stream, diaf_solve_info* info);

/* ---- Sparsified powers (Sec. 4.1, Algorithm 1) --------------------------------
 * The W pattern from the truncated Neumann series with the diagonal initial
 * subspace V_0: S = -D^-1 (A - D) (so that A = D (I - S); the structure does
 * not depend on the sign), per column s = t = e_j, then k times t = S t,
 * t dropped by count p_l, s = s + t; finally s dropped by count to `keep`
 * entries, the diagonal included.  Dropping by count keeps the p largest-
 * modulus off-diagonal entries (ties to the lower row; p_l <= 0 and keep <= 0
 * keep everything); the diagonal is never dropped and not counted; exact-zero
 * sums are not stored.  Sums are formed in a fixed order (row-sorted products,
 * separately rounded), so the pattern is reproducible.  A needs a zero-free
 * diagonal (DIAF_EINVAL otherwise); a column whose product list exceeds 512
 * entries gives DIAF_EUNSUPPORTED (use p_l).
 * Two calls: diaf_sparsified_count writes colptr (device, n + 1) and the
 * total to *nnz (host; synchronises `stream`); the caller allocates nnz rows
 * and diaf_sparsified_fill writes the sorted rows of every column. */
diaf_status diaf_sparsified_count(const diaf_csc* A, int32_t k, int32_t p_l, int32_t keep, int32_t* colptr,
                                  int64_t* nnz, void* stream);
/* Second pass of the sparsified-powers pattern (Sec. 4.1): writes the rows of
 * every column into rowidx (device, *nnz from the count) at colptr. */
diaf_status diaf_sparsified_fill(const diaf_csc* A, int32_t k, int32_t p_l, int32_t keep, const int32_t* colptr,
                                 int32_t* rowidx, void* stream);

/* ---- Learned proposal of the W pattern J_j ----------------------------------
 * Not in the paper: Sec. 4 chooses J_j by fixed rules (pattern(A), powers of
 * A, dropping by position).  Here a small network scores every candidate row
 * c of a candidate pattern CAND(:,j) (typically pattern(A^2)) and the best
 * ones are kept.  Features per candidate (DIAF_PROP_NFEAT floats, row-major
 * [CAND->nnz][8], in CAND's entry order):
 *   0 c == j   1 c is a row of A(:,j)   2 |A_cj| / max_i |A_ij|
 *   3 |(A^2)_cj| / max over CAND(:,j) of |(A^2)_c'j|
 *   4 log(|a_cc| / |a_jj|) clamped to [-10, 10] (0 if either is zero)
 *   5 |A_jc| / |a_jj|   6 nnz(A(:,c)) / nnz(A(:,j))   7 sign(j - c)
 * The network is 8 -> 32 -> 32 -> 1 with ReLU after both hidden layers;
 * parameters are DIAF_PROP_NPARAM floats: W1[32][8], b1[32], W2[32][32],
 * b2[32], w3[32], b3.  All pointers below are device pointers. */
#define DIAF_PROP_NFEAT 8
#define DIAF_PROP_HIDDEN 32
#define DIAF_PROP_NPARAM 1377

/* (Not in the paper: the learned proposal.)  Features of every entry of CAND
 * (same n as A, sorted columns of at most 128 rows -- pattern(A^3) of a
 * 7-point stencil has 63; DIAF_EUNSUPPORTED for a longer column) into feat
 * (device, [CAND->nnz][8]).  Synchronises `stream`.
 * Errors: EINVAL (NULL, sizes), EUNSUPPORTED, ECUDA. */
diaf_status diaf_propose_features(const diaf_csc* A, const diaf_pattern* CAND, float* feat, void* stream);

/* (Not in the paper.)  out[s] = network(feat[s]) for s < nrows (device
 * arrays).  Stream-ordered, allocates nothing.  Errors: EINVAL (NULL,
 * nrows < 0), ECUDA. */
diaf_status diaf_mlp_forward(const float* params, const float* feat, int64_t nrows, float* out, void* stream);

/* (Not in the paper.)
 * grad = d/dparams of loss = (1/nrows) sum_s (network(feat[s]) - target[s])^2,
 * *loss = that loss (both overwritten; grad has DIAF_PROP_NPARAM floats).
 * Per-block partial sums are added in block order: the result is reproducible.
 * Allocates (stream-ordered) one scratch row of DIAF_PROP_NPARAM + 1 floats
 * per 128 rows. */
diaf_status diaf_mlp_grad(const float* params, const float* feat, const float* target, int64_t nrows, float* grad,
                          float* loss, void* stream);

/* (Not in the paper.)  One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on
 * params with moment buffers m, v (DIAF_PROP_NPARAM device floats each, zero
 * before step 1); step >= 1 (EINVAL otherwise). */
diaf_status diaf_mlp_adam(float* params, const float* grad, float* m, float* v, int32_t step, float lr, void* stream);

/* (Not in the paper: the learned proposal's J_j, in place of the fixed rules
 * of Sec. 4.)  Keeps, per column j, min(keep, |CAND(:,j)|) rows: j itself
 * when it is a candidate, then the best scores (ties to the lower row; NaN
 * ranks last).
 * colptr (n+1) and rowidx (at most n*keep) are written; rows come out sorted.
 * Columns of CAND hold at most 128 rows (DIAF_EUNSUPPORTED otherwise; the
 * output is then incomplete).  Synchronises `stream`.  Errors: EINVAL (NULL,
 * keep < 1), ENOMEM, EUNSUPPORTED, ECUDA. */
diaf_status diaf_propose_select(const diaf_pattern* CAND, const float* score, int32_t keep, int32_t* colptr,
                                int32_t* rowidx, void* stream);

/* (Not in the paper: the training targets of the learned proposal.)
 * out[j] = res_j / |V(j,j)| for the factors F (infinity where V(j,j) is zero
 * or absent); with a diagonal V this is the norm of column j of
 * A W V^-1 - I.  out: n device doubles.  Stream-ordered, allocates nothing.
 * Errors: EINVAL (NULL), ECUDA. */
diaf_status diaf_scaled_residuals(const diaf_factors* F, double* out, void* stream);

/* (Not in the paper.)  Toggle targets of one candidate slot: for every
 * column j whose CAND column has an entry e at position `slot` other than
 * the diagonal, value[e] = L(rt_j) - L(r0_j) when in_base[e] != 0 (the
 * candidate was dropped from the base pattern) and L(r0_j) - L(rt_j)
 * otherwise (added), clipped to [-clip, clip], where r0 / rt are the scaled
 * residuals (diaf_scaled_residuals) of the base and of the toggled pattern,
 * L(r) = log(min(max(r^2, 1e-30 max(M, 1e-300)), 1e30 M)) with non-finite r
 * counted as the upper end, and M the largest finite r0_j^2 (1 when none is
 * positive).  Other entries of value are left as they are.  in_base:
 * CAND->nnz device bytes; r0, rt: n device doubles; value: CAND->nnz device
 * doubles.  Stream-ordered; allocates one scalar.  Errors: EINVAL (NULL,
 * slot < 0, clip <= 0), ENOMEM, ECUDA. */
diaf_status diaf_toggle_targets(const diaf_pattern* CAND, const uint8_t* in_base, const double* r0, const double* rt,
                                int32_t slot, double clip, double* value, void* stream);

/* Right-preconditioned restarted GMRES(restart) on A x = b (Sec. 5's solver
 * for the complex problems): x0 = 0, Arnoldi with classical Gram-Schmidt
 * applied twice, Givens rotations on the device, stop when the residual
 * estimate |g_{j+1}| <= tol ||b|| (the true residual is recomputed at every
 * restart), at most maxit inner iterations; 1 <= restart <= 64 (DIAF_EINVAL
 * otherwise).  F == NULL solves without preconditioner.  Allocates
 * (restart + 6) vectors of n scalars for the call.  info->breakdown is set
 * on a non-finite residual estimate. */
diaf_status diaf_gmres(diaf_solver* S, diaf_factors* F, const void* b, void* x, double tol, int32_t restart,
                       int32_t maxit, void* stream, diaf_solve_info* info);

/* Infrastructure: a static name for a status (never NULL), and the calling
 * thread's one-line reason for its last non-OK status ("" if none; valid
 * until that thread's next call). */
const char* diaf_status_string(diaf_status s);
const char* diaf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DIAF_H */
