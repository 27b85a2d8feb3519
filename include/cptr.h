/*
 * cptr.h -- C ABI of the GB300 (sm_103a) CPTR-FGMRES library.
 *
 * Solves one Newton linear system A dx = b of fully implicit non-isothermal multiphase porous-
 * media flow with right-preconditioned flexible GMRES and the two-stage Constrained Pressure-
 * Temperature Residual preconditioner of Roy, Jonsthovel, Lemon, Wathen (arXiv 1907.04229):
 *   Sec. 3.2, eq. (AXR)     the block system in (p, T, saturations) unknowns;
 *   Sec. 2.2.2, eqs. (weighted), (scaling)   equation weighting applied as A' = W A, b' = W b;
 *   Sec. 3, "Two-stage preconditioners"     z = M2^{-1}(v - A' x1) + x1, x1 = M1^{-1} v;
 *   Sec. 3.2 eq. (A00), Sec. 3.3 eq. (Aschur) and its five steps    stage 1 on the p-T block;
 *   Sec. 3.3.1 eq. (Se)     the Schur-complement approximation S~_T (supplied by the caller);
 *   Sec. 3.1                CPR (pressure-only first stage), the baseline;
 *   Sec. 4                  ILU(0) second stage, AMG V-cycles for A_pp and S~_T, GMRES tol.
 * Every step runs in this library's CUDA kernels on the current device.  All calls are
 * synchronous with respect to the host unless stated otherwise.
 *
 * Conventions for every entry point:
 *   - Return value: CPTR_OK (0), CPTR_NOT_CONVERGED (1) or a negative error code.  No C++
 *     exception crosses the ABI.  After an error, cptr_last_error(ctx) describes it.
 *   - Ownership: the caller owns every input and output buffer.  The library copies what it
 *     keeps; nothing the caller passes is retained after a call returns.
 *   - Pointers: "on_device" = 1 means every array argument of the call is device memory of the
 *     current device (e.g. a torch CUDA tensor's data_ptr); 0 means host memory, copied inside.
 *   - Indices are int32, values IEEE double, arrays contiguous.
 */
#ifndef CPTR_H
#define CPTR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cptr_ctx cptr_ctx;

typedef enum {
    CPTR_OK = 0,
    CPTR_NOT_CONVERGED = 1, /* max_it reached; x holds the last iterate, stats are filled */
    CPTR_EINVAL = -1,       /* invalid argument or malformed matrix (message says which) */
    CPTR_ENOMEM = -2,       /* device allocation failed */
    CPTR_ECUDA = -3,        /* a CUDA runtime call failed */
    CPTR_EBREAKDOWN = -4,   /* non-finite value in the Krylov iteration */
    CPTR_ETIMEOUT = -5,     /* a bounded device-side wait gave up */
    CPTR_ESINGULAR = -6,    /* zero pivot in ILU(0) or singular coarsest AMG matrix */
    CPTR_ESTATE = -7,       /* call out of order (e.g. solve before setup) */
    CPTR_ECHECK = -8        /* bounds-checking build (libcptr_check.so) only: an index read from a
                             * table on the device fell outside its array; the access was skipped,
                             * and the message names the kernel site, the index and the bound */
} cptr_status;

/* first stage M1 (Sec. 3.1, 3.3, 3.4): full block factorisation, its block-triangular variants
 * (one factor of eq. (Aschur) dropped), block diagonal, CPR pressure-only, none, or one V-cycle of
 * unknown-based AMG on A_00 (Sec. 3.4: classical coarsening and direct interpolation of the A_pp
 * and A_TT diagonal blocks on their own, with PMIS weights indexed within each block; the Galerkin
 * product and the smoother on the whole coupled A_00 in unknown-wise order [p; T], so the coupling
 * blocks stay in the coarse-grid correction; the Schur approximation is not used) */
enum { CPTR_STAGE1_FULL = 0, CPTR_STAGE1_UPPER = 1, CPTR_STAGE1_LOWER = 2, CPTR_STAGE1_BD = 3,
       CPTR_STAGE1_CPR = 4, CPTR_STAGE1_NONE = 5, CPTR_STAGE1_UAMG = 6 };
/* second stage M2: ILU(0) on the full system (Sec. 4) or none */
enum { CPTR_STAGE2_ILU0 = 0, CPTR_STAGE2_NONE = 1 };
/* Schur approximation: the caller's S~_T (eq. Se) or A_TT (Sec. 3.3.1), the learned diagonal
 * scaling diag(s) B of B = the caller's S~_T, else A_TT (see cptr_set_mlp; not in the paper), or
 * S~_diag = A_TT - A_Tp diag(A_pp)^{-1} A_pT (Sec. 3.3.1), formed on the device on its own pattern
 * (A_TT's joined with that of the product): the product column-scales A_Tp by 1 / (A_pp)_kk and
 * sums every entry over k ascending with separately rounded products and sums */
enum { CPTR_SCHUR_GIVEN = 0, CPTR_SCHUR_ATT = 1, CPTR_SCHUR_LEARNED = 2, CPTR_SCHUR_DIAG = 3 };
/* AMG smoother: l1-Jacobi (d_i = sum_j |a_ij|) or omega-Jacobi (d_i = a_ii / omega) */
enum { CPTR_SMOOTH_L1 = 0, CPTR_SMOOTH_JACOBI = 1 };
/* precision of the preconditioner: all FP64, or FP32 AMG/ILU with BF16 coarse AMG levels */
enum { CPTR_PREC_FP64 = 0, CPTR_PREC_MIXED = 1 };
/* cell order of the ILU(0) factorisation (the paper does not state one): the caller's order, or
 * multicolour: greedy distance-1 colouring of the cell graph in the caller's order, cells sorted
 * by (colour, index) -- red-black on a 7-point grid, two level sets per triangular sweep */
enum { CPTR_ILU_NATURAL = 0, CPTR_ILU_MULTICOLOR = 1 };
/* decoupling operator G = [I -D; 0 I] of the first stage, applied inside it: M1^{-1} =
 * R^T (R G A' R^T)^{-1} R G (Sec. 3.1), i.e. stage 1 solves with A_pp - D A_sp (CPR) or A_00 - D A_s0
 * (p-T first stage, Sec. 3.2) on the right-hand side R G v; the system and the second stage keep A'.
 * D is block diagonal, D_i = X_i Y_i^{-1}: Quasi-IMPES takes X_i, Y_i from the cell's diagonal block
 * (primary rows x secondary columns, secondary x secondary), True-IMPES from the sum of the blocks
 * of block column i (the pattern must then be structurally symmetric).  Y_i^{-1} by Gauss-Jordan
 * with partial pivoting; primary slots {p} for CPR, {p, T} otherwise. */
enum { CPTR_DECOUPLE_NONE = 0, CPTR_DECOUPLE_QI = 1, CPTR_DECOUPLE_TI = 2 };
/* unknown kinds, one per block slot */
enum { CPTR_U_P = 0, CPTR_U_T = 1, CPTR_U_SAT = 2 };

typedef struct {
    int32_t stage1, stage2, schur, smoother;
    double omega;        /* omega-Jacobi weight (default 2/3) */
    double theta;        /* AMG strength threshold (default 0.25) */
    int32_t n_coarse;    /* stop coarsening at n <= n_coarse (default 256) */
    int32_t max_levels;  /* AMG levels including the coarsest (default 25) */
    int32_t restart;     /* FGMRES restart length m (default 30, at most 32) */
    int32_t max_it;      /* total Arnoldi steps (default 1000) */
    int32_t dense_max;   /* coarsest level solved densely if n <= dense_max (default 1024, at most 25600) */
    int32_t seed;        /* PMIS weights: SplitMix64 stream seed + level */
    int32_t precision;   /* CPTR_PREC_* */
    int32_t check_every; /* host reads the convergence flag every k Arnoldi steps (default 1) */
    int32_t use_graph;   /* 1 (default): each FGMRES restart cycle is one captured CUDA graph whose
                          * conditional WHILE node repeats the Arnoldi step on the device until the
                          * cycle ends (the host waits once per cycle); 2: one captured graph launch
                          * per Arnoldi step (the host checks convergence after each); 0: direct
                          * kernel launches.  Solves with per-family profiling or wait injection on
                          * use per-step graphs. */
    int32_t ilu_order;   /* CPTR_ILU_NATURAL (default) or CPTR_ILU_MULTICOLOR */
    int32_t autotune;    /* 1: time the launch shapes of the V-cycle and SpMV kernels at set-up
                            and keep the fastest (see cptr_tuning); 0 (default): fixed shapes */
    int32_t ilu_sweep;   /* schedule of the ILU(0) triangular sweeps: 0 (default) level sets, or,
                            with autotune, the fastest of level sets, grouped levels, the chunked
                            wavefront and tiles where the pattern allows them; 1 level sets;
                            2 chunked wavefront (natural order, at most 4 dependencies per row,
                            levels no wider than 256 rows inside a chunk; same values as level
                            sets); 3 grouped levels (ilu_group levels per group, two by default:
                            paired levels), else level sets (a row substitutes its dependencies
                            inside its group, so the group's levels run as one; values differ from
                            level sets by rounding); 4 tiles where the pattern is that
                            of a Cartesian box in natural order (lower dependencies at offsets 1,
                            nx and nx*ny only), else level sets: a block owns a tile of Ty x Tz
                            grid lines and walks the tile's own level sets, only dependencies on
                            other tiles crossing blocks (same values as level sets) */
    void *stream;        /* cudaStream_t for all work; NULL = the legacy default stream */
    int32_t tile_y;      /* tiled sweeps (ilu_sweep 4): grid lines per tile along y and z; 0 (default):
                            the shape of smallest modelled time, or with autotune the fastest of the
                            four best modelled ones */
    int32_t tile_z;
    int32_t decouple;    /* decoupling operator of the first stage (Sec. 3.1, extended to the p-T system
                            in Sec. 3.2): CPTR_DECOUPLE_NONE (default), _QI or _TI; for the CPR and
                            unknown-based first stages only (the Schur approximation of the block
                            preconditioner cannot be combined with it, Sec. 3.3.1) */
    int32_t ilu_fill;    /* level of fill of the second stage's block ILU(k): 0 (default) or 1 (block row
                            i gains, for every block k < i of its row, the blocks j > k of row k;
                            natural ILU order only; the sweeps then use level sets or grouped levels) */
    int32_t csr_lanes;   /* lanes per row of the V-cycle kernels (smoother + residual, restriction,
                            prolongation) on every level when autotune is 0: 0 (default) chosen from
                            each operator's size and average row length, else 1, 2, 4, 8, 16 or 32
                            (other values: CPTR_EINVAL at cptr_create).  One lane adds a row's
                            products in order; more lanes add lane-strided partial sums. */
    int32_t ilu_group;   /* levels per group of the grouped-level sweeps (ilu_sweep 3, or the autotuner's
                            grouped-level candidate): 0 (default) two, or 2, 3 or 4.  A row
                            of a group substitutes the equations of its dependencies inside the group
                            (chains of up to group - 1 links), so the sweep's dependent steps are the
                            level count divided by the group size; values differ from level sets by
                            rounding.  When a row's expansion has more than 32 dependencies (or 32
                            right-hand-side terms) the tables are not built and level sets are used
                            (other values: CPTR_EINVAL at cptr_create). */
    int32_t ilu_lanes;   /* lanes per row of the grouped-level sweeps: 0 (default) four, or with
                            autotune the fastest of 4, 8 and 16; 4, 8 or 16 fixes it.  Four lanes:
                            lane q computes component q over all of the row's dependency slots; 8 or
                            16: H = 2 or 4 parts of four lanes each take every H-th slot, and their
                            partial sums are added pairwise at the end, which shortens each lane's
                            chain of FP64 instructions to about 1/H; values differ by rounding (other
                            values: CPTR_EINVAL at cptr_create). */
} cptr_options;

typedef struct {
    int32_t iters;           /* Arnoldi steps taken (all restart cycles) */
    int32_t restarts;
    int32_t converged;
    int32_t levels_p, levels_T;
    int32_t schur_used;      /* S~_T the set-up used: CPTR_SCHUR_GIVEN, _ATT or _LEARNED */
    double est_rel_res;      /* Givens estimate |g_{j+1}| / ||b'|| at exit */
    double true_rel_res;     /* ||b' - A' x|| / ||b'|| recomputed at exit */
    double bnorm;            /* ||b'|| = ||W rhs|| */
    double setup_ms, solve_ms;
    double op_complexity_p, op_complexity_T;
} cptr_stats;

/* Fill *opt with the defaults listed above. */
cptr_status cptr_default_options(cptr_options *opt);

/* Create a context on the current device.  *out receives it (NULL on failure). */
cptr_status cptr_create(cptr_ctx **out, const cptr_options *opt);

/* Destroy a context and free its device memory (NULL is ignored). */
void cptr_destroy(cptr_ctx *ctx);

/* Message of the last error on ctx ("" if none).  Valid until the next call on ctx. */
const char *cptr_last_error(const cptr_ctx *ctx);

/*
 * Set up the preconditioner for one Jacobian (Sec. 3.2 eq. AXR; Sec. 3.3; Sec. 4).
 *   n_cells, b     number of cells and unknowns per cell (b = 3 or 4)
 *   row_ptr        [n_cells+1] BSR block-row pointers
 *   col_idx        [nnzb] block column indices, strictly ascending within each row, the
 *                  diagonal block present in every row
 *   vals           [nnzb*b*b] raw Jacobian blocks, row-major within a block:
 *                  vals[(k*b + r)*b + c] = d(equation r)/d(unknown c) of block k
 *   unknown_kind   [b] CPTR_U_* per slot; exactly one P and one T
 *   row_weights    [n_cells*b*b] per-cell W_i (row-major), the decoupled block row is W_i times
 *                  the raw block row (eqs. weighted, scaling); NULL = identity
 *   st_vals        [nnzb] S~_T on the same cell pattern (eq. Se); NULL = A_TT
 * Validates the pattern on the host and the values on the device (finite), then builds on the
 * device: the decoupled A', the p-T blocks, two AMG hierarchies and the ILU(0) factors.
 * Errors: CPTR_EINVAL (bad sizes or pattern, non-finite values), CPTR_ESINGULAR, CPTR_ENOMEM,
 * CPTR_ECUDA.  A context may be set up again; the previous setup is released first.
 */
cptr_status cptr_setup(cptr_ctx *ctx, int32_t n_cells, int32_t b, const int32_t *row_ptr,
                       const int32_t *col_idx, const double *vals, const int32_t *unknown_kind,
                       const double *row_weights, const double *st_vals, int32_t on_device);

/*
 * Solve A' x = W rhs with FGMRES(m) from x = 0 until |g_{j+1}| <= rtol * ||W rhs|| (Sec. 4).
 *   rhs  [n_cells*b] raw right-hand side (cell-major, slot order of the setup)
 *   x    [n_cells*b] output solution
 *   st   optional statistics (may be NULL)
 * Returns CPTR_OK, CPTR_NOT_CONVERGED (x = last iterate), CPTR_EBREAKDOWN, CPTR_ETIMEOUT,
 * CPTR_ESTATE (no setup) or CPTR_ECUDA.
 */
cptr_status cptr_solve(cptr_ctx *ctx, const double *rhs, double *x, double rtol, cptr_stats *st,
                       int32_t on_device);

/*
 * Block-Jacobi second stage (Sec. 4: in parallel the paper applies ILU(k) to each block of the
 * domain's partition across processes, "block Jacobi"): with a partition set, the ILU(0) factors
 * drop every coupling between cells of different parts, so each part is factored and solved on
 * its own.  This is the paper's second stage for that many processes, in one solve.
 *   part  [n_cells] part id of every cell (any int32 values; cells with equal ids form a part);
 *         NULL removes the partition (global ILU(0), the default)
 * Copied into context memory (host or device pointer, on_device as in cptr_setup); takes effect at
 * the next cptr_setup, whose n_cells must equal n_cells here.  Natural order and ILU(0) only:
 * that set-up returns CPTR_EINVAL with the multicolour order or ILU(1); the chunked and tiled sweep
 * schedules are not used with a partition.  Errors: CPTR_EINVAL, CPTR_ENOMEM, CPTR_ECUDA.
 */
cptr_status cptr_set_partition(cptr_ctx *ctx, int32_t n_cells, const int32_t *part, int32_t on_device);

/* ------------------------------------------------------------------------------------------
 * Component entry points.  They apply one piece of the set-up operator, for parity tests and
 * profiling.  All vectors are device memory of length n_cells*b (cell-major) unless stated.
 * ------------------------------------------------------------------------------------------ */

/* y = A' x with the decoupled Jacobian A' = W A (BSR SpMV). */
cptr_status cptr_apply_matrix(cptr_ctx *ctx, const double *x, double *y);

/* out = W rhs (per-cell b x b weights). */
cptr_status cptr_apply_weights(cptr_ctx *ctx, const double *rhs, double *out);

/* x1 = M1^{-1} v: stage 1 of the selected kind; slots other than p and T are set to 0. */
cptr_status cptr_apply_stage1(cptr_ctx *ctx, const double *v, double *x1);

/* z = (L U)^{-1} r with the block ILU(0) factors of A'. */
cptr_status cptr_apply_ilu(cptr_ctx *ctx, const double *r, double *z);

/* z = M^{-1} v, the full two-stage preconditioner. */
cptr_status cptr_apply_precond(cptr_ctx *ctx, const double *v, double *z);

/* x = one V(1,1)-cycle from zero on hierarchy `which` (0: A_pp, 1: S~_T); b, x of length n_cells.
 * With CPTR_STAGE1_UAMG, hierarchy 0 is the unknown-based one of A_00 and b, x have length 2 n_cells
 * ([p; T], unknown-wise). */
cptr_status cptr_apply_vcycle(cptr_ctx *ctx, int32_t which, const double *b, double *x);

/* Hierarchy shape: *nlev levels; for level l, info[l*4 + {0,1,2,3}] = {n, nnz, nnzP, dense}
 * (nnzP = 0 on the coarsest level; dense = 1 if the coarsest level is solved densely).
 * info must hold 4 * 32 int32 (host memory). */
cptr_status cptr_hierarchy_info(cptr_ctx *ctx, int32_t which, int32_t *nlev, int32_t *info);

/* Copy level l of hierarchy `which` to host buffers sized from cptr_hierarchy_info:
 * rp[n+1], ci[nnz], v[nnz], dinv[n]; and if l is not the coarsest: cf[n] (1 = C, 2 = F),
 * Prp[n+1], Pci[nnzP], Pv[nnzP].  Any pointer may be NULL to skip that array. */
cptr_status cptr_hierarchy_level(cptr_ctx *ctx, int32_t which, int32_t l, int32_t *rp, int32_t *ci,
                                 double *v, double *dinv, int32_t *cf, int32_t *Prp, int32_t *Pci,
                                 double *Pv);

/* z = (L U)^{-1} r with the block ILU(0) factors of A', for callers that cannot allocate device
 * memory when they apply the preconditioner: code running while a framework's caching allocator
 * owns the whole device, real-time loops that cannot pay for cudaMalloc/cudaFree (cudaFree also
 * synchronises the device), or deployments whose memory budget is fixed in advance.  The call
 * allocates nothing and does not use the context's work vectors: the two intermediate vectors of
 * the triangular solves live in one file-scope device array of 2 x 2^20 doubles (16 MiB), which
 * every GPU that loads the library keeps until the process exits.  The paper has no counterpart;
 * it is an engineering addition.
 *   r, z   device vectors of n_cells*b doubles; n_cells*b must not exceed 2^20, else
 *          CPTR_EINVAL with a message naming the limit.  Natural ILU ordering and ILU(0) only
 *          (else CPTR_EINVAL).
 * It always applies the FP64 factors (one launch per level set), also in a context of the mixed
 * precision or with another sweep schedule, so its result equals cptr_apply_ilu of an FP64
 * context to rounding.  The array's device address is looked up with the call's device current,
 * on every call whose stream is not being captured; the first call on a device does that set-up
 * and must come before any stream capture.  All calls on a device share the array: calls whose
 * work overlaps on the GPU race on it.  No part of the array needs to start at zero (each call
 * writes every element it later reads).  The call synchronises the context's stream before it
 * returns.  Errors: CPTR_ESTATE (no setup, no ILU(0), or a first call under capture),
 * CPTR_EINVAL, CPTR_ECUDA. */
cptr_status cptr_apply_ilu_static(cptr_ctx *ctx, const double *r, double *z);

/* Launch shapes in use (an engineering addition; the paper has none).  Writes up to cap rows of 5
 * int32 into rows (host): {hierarchy (0 A_pp, 1 S~_T, 2 A', 3 ILU(0)), level, kernel (0 smoother +
 * residual, 1 restriction P^T, 2 prolongation P, 3 SELL SpMV of A', 4 ILU(0) sweeps, 5 ILU(0)
 * schedule, 6 tile shape of the tiled sweeps, 7 lanes per row of the grouped-level sweeps), lanes
 * per row (0 = chosen from the average row length; kernel 4: back-off between polls in ns;
 * kernel 5: 0 level sets, 1 chunked wavefront, 2 grouped levels, 3 tiles; kernel 6: lines per tile
 * along y, Ty, or 0 when no tiled tables are built; kernel 7: 4, 8 or 16, or 0 when the grouped levels
 * are not in use), threads per block (kernel 4: blocks of the persistent grid; kernel 5: levels
 * per group of the grouped levels, else 0; kernel 6: lines per tile along z, Tz)}; *n_rows
 * receives the number of rows available.  With autotune set,
 * cptr_setup times for every operator G in {1, 2, 4, 8, 16, 32} lanes x T in {128, 256, 512}
 * threads (the SELL kernels: T in {64, 128, 256, 512}), 5 launches each after a warm-up, and keeps
 * the fastest; results are cached in the context by operator size.  Shapes change only the order
 * of the partial sums within a row.  Errors: CPTR_ESTATE, CPTR_EINVAL. */
cptr_status cptr_tuning(cptr_ctx *ctx, int32_t *rows, int32_t cap, int32_t *n_rows);

/* Number of ILU level sets of the forward and backward sweeps (host ints). */
cptr_status cptr_ilu_levels(cptr_ctx *ctx, int32_t *n_forward, int32_t *n_backward);

/* Failure injection for tests (no GPU fault involved): while on != 0, the first row of every
 * forward ILU(0) sweep also waits for a value that no thread ever writes.  The bounded wait gives
 * up after about 0.5 s, the sweep completes, and the call (cptr_solve, cptr_apply_ilu,
 * cptr_apply_precond) returns CPTR_ETIMEOUT.  The context stays usable; switch it off to solve
 * normally again.  The paper has no counterpart; it exercises the library's own wait limits. */
cptr_status cptr_inject_wait_timeout(cptr_ctx *ctx, int32_t on);

/* Number of kernels this library has launched in this process (all contexts, since load). */
int64_t cptr_launch_count(void);

/* Time families of kernels with CUDA events on the context's stream during cptr_solve; bit f
 * of mask enables family f: 0 the outer SpMV w = A' z_j (one kernel per region), 1 stage 1,
 * 2 the stage-1 residual v - A' x1 (one kernel), 3 the ILU(0) solve (three kernels), 4 Arnoldi
 * (three Gram-Schmidt passes, Givens, normalisation), 5 the forward ILU sweep (one kernel),
 * 6 the backward ILU sweep (one kernel); bit 7 times each kernel of the finest level of the
 * V-cycles one by one (read by cptr_profile_vcycle).  0 disables (the default). */
cptr_status cptr_set_profiling(cptr_ctx *ctx, uint32_t mask);

/* Event time (ms) and number of timed regions per family during the last cptr_solve (host
 * arrays of 16 entries; either may be NULL): entries 0-7 the families above; entries 8-15 the
 * host-clock time of the last cptr_setup's phases, with count 1: 8 inputs + decoupling +
 * extraction, 9 AMG coarsening (strength, PMIS, interpolation), 10 AMG Galerkin products,
 * 11 AMG coarsest inverses, 12 ILU host work (ordering, level sets, sweep tables), 13 ILU
 * factorisation, 14 SELL layout and mixed-precision copies, 15 other. */
cptr_status cptr_profile(cptr_ctx *ctx, double *ms, int64_t *count);

/* Event time (ms) and number of launches of the finest AMG level's V(1,1)-cycle kernels during the
 * last cptr_solve with bit 7 of the profiling mask set (host arrays of 8 entries; either may be
 * NULL).  Entry 4*h + k: hierarchy h (0 the pressure hierarchy, or the p-T one of the
 * unknown-based first stage; 1 the temperature hierarchy of S~_T), kernel k: 0 pre-smoothing from
 * zero fused with the residual (t = D^-1 b, r = b - A t), 1 restriction b_c = P^T r,
 * 2 prolongation t += P x_c, 3 post-smoothing x = t + D^-1 (b - A t) (Sec. 3.3: the V-cycles of
 * the first stage).  A fine level whose kernels are fused with the coarse ones (at most a few
 * hundred rows) is not timed. */
cptr_status cptr_profile_vcycle(cptr_ctx *ctx, double *ms, int64_t *count);

/* ---------------------------------------------------------------------------------------------
 * Ensemble: many independent Jacobians (realisations of a model, of uneven sizes) set up and
 * solved together.  The paper solves one system at a time; this extension follows its method per
 * instance.  The instances are set up as ONE block-diagonal system (instance k = a consecutive
 * range of cells), so the AMG hierarchies, ILU(0) factors and SpMVs are built and applied on the
 * union with one launch per kernel, and every block of them acts on its own instance only (the
 * strength graph, interpolation, Galerkin products, ILU(0) pattern and coarsest inverse of a
 * block-diagonal matrix are block diagonal).  PMIS weights use the union's cell index, so an
 * instance's coarse grids are not those of a separate set-up; coarsening continues while the union
 * has more than n_coarse points.  FGMRES runs per instance: its own Krylov basis, Givens rotations
 * and stopping test |g_{j+1}| <= rtol ||W_k rhs_k||.  All instances take Arnoldi steps in lockstep
 * (one captured CUDA graph per step for the whole ensemble); an instance that has converged is
 * skipped by the Gram-Schmidt kernels, keeps its solution, and its step count stops.
 * --------------------------------------------------------------------------------------------- */
typedef struct {
    int32_t n_cells;
    const int32_t *row_ptr, *col_idx;  /* BSR pattern of the instance, 0-based within it */
    const double *vals;                /* [nnzb][b][b] */
    const double *row_weights;         /* [n_cells][b][b] or NULL (NULL for all or for none) */
    const double *st_vals;             /* S~_T on the instance's pattern or NULL (all or none) */
} cptr_instance;

/* Set up n_inst instances with the same b and unknown_kind (all arrays host or device per
 * on_device; unknown_kind likewise).  Replaces any previous set-up of ctx.  Errors as cptr_setup,
 * and CPTR_EINVAL when only some instances give row_weights or st_vals. */
cptr_status cptr_setup_batch(cptr_ctx *ctx, int32_t n_inst, int32_t b, const cptr_instance *inst,
                             const int32_t *unknown_kind, int32_t on_device);

/* Solve every instance to its own relative residual rtol: rhs[k] and x[k] (host arrays of n_inst
 * pointers to n_cells_k * b doubles each, host or device memory per on_device); x[k] is
 * overwritten.  st: host array of n_inst stats (iters and restarts per instance; setup_ms and
 * solve_ms are the whole ensemble's), may be NULL.  Returns CPTR_OK when all converged,
 * CPTR_NOT_CONVERGED when some reached max_it total Arnoldi steps; other errors as cptr_solve.
 * Errors: CPTR_ESTATE when the last set-up was not cptr_setup_batch. */
cptr_status cptr_solve_batch(cptr_ctx *ctx, const double *const *rhs, double *const *x, double rtol,
                             cptr_stats *st, int32_t on_device);

/* ---------------------------------------------------------------------------------------------
 * Learned diagonal scaling of the Schur approximation.  The paper has no learned part: it
 * approximates S_T = A_TT - A_Tp A_pp^{-1} A_pT by the discrete S_e or, without it, by A_TT
 * (Sec. 3.3.1).  This extension scales the rows of that base approximation B (st_vals when the
 * caller gives them, else A_TT): S~_T = diag(s) B with s_i = sinh(y_i), where y_i is the output of
 * a 16-64-64-1 tanh network over 16 local features of cell i of A'.  It is meant to be trained on
 * asinh((S_T)_ii / B_ii) computed exactly on small grids.
 *
 * Features of cell i (all sums over the pattern of row i in ascending order; B as above;
 * q(x, y) = x / y, or 0 when y = 0; a = the diagonal b x b block of A'; s over saturation slots;
 * every value v is stored as asinh(v)):
 *   0  q(sum_j A_Tp,ij q(A_pT,ji, A_pp,jj), B_ii)   1  q(A_Tp,ii q(A_pT,ii, A_pp,ii), B_ii)
 *   2  q(sum_{j!=i} |A_pp,ij|, |A_pp,ii|)           3  q(sum_{j!=i} |B_ij|, |B_ii|)
 *   4  q(sum_{j!=i} A_pp,ij, |A_pp,ii|)             5  q(sum_{j!=i} B_ij, |B_ii|)
 *   6  q(sum_j |A_Tp,ij q(A_pT,ji, A_pp,jj)|, |B_ii|)
 *   7  q(sum_s a_Ts q(a_sT, a_ss), B_ii)            8  q(sum_s a_ps q(a_sp, a_ss), A_pp,ii)
 *   9  sign(A_pp,ii)                                10 sign(B_ii)
 *   11 q(A_pT,ii, sqrt|A_pp,ii B_ii|)                12 q(A_Tp,ii, sqrt|A_pp,ii B_ii|)
 *   13 (entries in row i) / 7
 *   14 q(sum_{j!=i} |A_pT,ij| |A_Tp,ii|, |A_pp,ii B_ii|)
 *   15 q(sum_{j!=i} |A_Tp,ij| |A_pT,ii|, |A_pp,ii B_ii|)
 * A_pT,ji is 0 when the pattern has no entry (j, i).
 *
 * Parameters: CPTR_MLP_NPARAM floats, W1[64][16] | b1[64] | W2[64][64] | b2[64] | w3[64] | b3;
 * z1 = W1 x + b1, h1 = tanh z1, z2 = W2 h1 + b2, h2 = tanh z2, y = w3 . h2 + b3.
 * Training: FP32, mean squared error (1/n) sum (y_i - t_i)^2, full-batch Adam (beta1 0.9,
 * beta2 0.999, eps 1e-8) from zero moments.  Inference (set-up): BF16 weights and layer inputs
 * (features FP64 -> FP32 -> BF16, round to nearest even), FP32 biases, each layer's sum
 * accumulated in FP32 from the bias in ascending input order, tanh in FP32.
 * ------------------------------------------------------------------------------------------- */
#define CPTR_MLP_FEATURES 16
#define CPTR_MLP_HIDDEN 64
#define CPTR_MLP_NPARAM 5313

/* Features of every cell of the current set-up into feat[n_cells][16] (FP64, host or device per
 * on_device).  Errors: CPTR_ESTATE (no set-up), CPTR_EINVAL, CPTR_ECUDA. */
cptr_status cptr_schur_features(cptr_ctx *ctx, double *feat, int32_t on_device);

/* Loss and gradient of the network at params over n samples: feat[n][16], target[n] (FP64,
 * rounded to FP32 on the device), params[CPTR_MLP_NPARAM] and grad[CPTR_MLP_NPARAM] (FP32),
 * *loss (host double, may be NULL).  All arrays host or device per on_device.  Needs no set-up.
 * Errors: CPTR_EINVAL (n < 1, null arrays), CPTR_ENOMEM, CPTR_ECUDA. */
cptr_status cptr_mlp_loss_grad(cptr_ctx *ctx, const double *feat, const double *target, int32_t n,
                               const float *params, float *grad, double *loss, int32_t on_device);

/* Train in place: params (FP32, in: initial, out: trained) after `steps` full-batch Adam steps
 * with learning rate lr.  loss_hist[steps] (host doubles, may be NULL) receives the loss before
 * each step.  Arrays host or device per on_device (loss_hist always host).  Needs no set-up.
 * Errors: CPTR_EINVAL, CPTR_ENOMEM, CPTR_ECUDA. */
cptr_status cptr_mlp_train(cptr_ctx *ctx, const double *feat, const double *target, int32_t n, float *params,
                           int32_t steps, float lr, double *loss_hist, int32_t on_device);

/* Give the context a network for CPTR_SCHUR_LEARNED (params copied; NULL removes it).  A set-up
 * with CPTR_SCHUR_LEARNED and no network, or whose s is not finite or has |y| > 30 anywhere,
 * falls back to the caller's S~_T if st_vals was given, else to A_TT; cptr_stats.schur_used
 * reports which.  Errors: CPTR_EINVAL, CPTR_ECUDA. */
cptr_status cptr_set_mlp(cptr_ctx *ctx, const float *params, int32_t on_device);

/* BF16 inference of the context's network on feat[n][16] (FP64) into y[n] (FP32).  Errors:
 * CPTR_ESTATE (no network), CPTR_EINVAL, CPTR_ENOMEM, CPTR_ECUDA. */
cptr_status cptr_mlp_infer(cptr_ctx *ctx, const double *feat, int32_t n, float *y, int32_t on_device);

/* The row scaling s[n_cells] of the last set-up (all ones unless it used the learned form).
 * Features (cptr_schur_features) always refer to the unscaled base B.
 * Errors: CPTR_ESTATE, CPTR_EINVAL, CPTR_ECUDA. */
cptr_status cptr_schur_scaling(cptr_ctx *ctx, double *s, int32_t on_device);

/* ---------------------------------------------------------------------------------------------
 * Newton's method around the solve (Sec. 3 eq. (AXR): every Newton iteration solves J dx = -R with
 * the context's CPTR-FGMRES; Sec. 4: Newton with line search, tolerance 1e-8 on the relative
 * function norm and on the relative step norm), with the residual, Jacobian and S_e assembled on
 * the device for the thermal multiphase finite-volume model of Sec. 2 on an nx x ny x nz Cartesian
 * box in natural cell order (x fastest).  Unknowns per cell (p, T, S_w[, S_g]) in Pa, K and
 * fractions; raw equation rows water mass, energy, oil mass[, gas mass] (kg/s, W).  TPFA with
 * harmonic K and k_T, arithmetic face density, phase upwinding on the potential difference (ties to
 * the lower-index cell), implicit Euler; water density and viscosity by the correlations of
 * Appendix A; oil density rho_o_ref exp(c_o (p - p0) - beta_o (T - T0)), oil viscosity
 * mu_o_ref exp(-beta_mu (T - T0)), ideal gas of molar mass gas_M and viscosity mu_g; Corey k_r =
 * max(S, 0)^corey_n; k_T = kT_const if > 0, else (1 - phi) kT_rock + phi sum_alpha S_alpha kT_alpha.
 * Wells: kind 0 injects water at rate a (m^3/s) and temperature c (K); kind 1 produces each phase at
 * q_alpha = a lam_alpha (p - c)^+ (a = WI in m^3, c = bottom-hole pressure).  Heaters add
 * U (T_heater - T) to the energy equation.  S_e (eq. Se): the energy equation with every
 * coefficient frozen at the iterate, differentiated in the explicit temperature factors only.
 * --------------------------------------------------------------------------------------------- */
typedef struct {
    int32_t nx, ny, nz, nphase;   /* nphase 2 (b = 3) or 3 (b = 4) */
    double dx, dy, dz;            /* cell sizes, m; depth grows with z */
    double dt, phi, grav;         /* time step (s), porosity, gravity (m/s^2) */
    const double *kh, *kv;        /* [n] permeability, m^2: x and y faces use kh, z faces kv */
    double kT_const, kT_rock, kT_w, kT_o, kT_g;         /* W/m/K */
    double cv_w, cv_o, cv_g, c_rock, rho_rock;          /* J/kg/K, kg/m^3 */
    double mu_o_ref, beta_mu, T0, rho_o_ref, c_o, beta_o, p0;
    double gas_M, mu_g, corey_n;
    int32_t n_wells, n_heaters;
    const int32_t *well_cell, *well_kind;   /* [n_wells] */
    const double *well_a, *well_c;          /* [n_wells] */
    const int32_t *heater_cell;             /* [n_heaters] */
    const double *heater_U, *heater_T;      /* [n_heaters] W/K, K */
    const double *weights;                  /* [n][b][b] equation weights W of the solve (NULL: identity) */
} cptr_model;

typedef struct {
    int32_t newton_its, linear_its, line_search_cuts, converged;
    double res0, res;             /* ||W R|| at the start and at the end */
    double setup_ms, solve_ms;    /* summed over the Newton iterations */
} cptr_newton_stats;

/* Give the context a model (copied; its arrays host or device per on_device).  Errors: CPTR_EINVAL,
 * CPTR_ENOMEM, CPTR_ECUDA. */
cptr_status cptr_model_set(cptr_ctx *ctx, const cptr_model *model, int32_t on_device);

/* Residual R(x) ([n][b] raw rows) of the implicit Euler step from xn to x, and if J / Se are not NULL
 * the analytic Jacobian dR/dx ([nnzb][b][b], row-major blocks) and S_e ([nnzb]) on the 7-point
 * pattern (rows in natural order, columns ascending).  One thread per cell gathers its rows: its
 * accumulation terms, its wells and heaters in the caller's order, then its faces (i - nx ny, i),
 * (i - nx, i), (i - 1, i), (i, i + 1), (i, i + nx), (i, i + nx ny), every product and sum rounded on
 * its own.  Arrays host or device per on_device.  Errors: CPTR_ESTATE (no model), CPTR_EINVAL. */
cptr_status cptr_assemble(cptr_ctx *ctx, const double *x, const double *xn, double *R, double *J, double *Se,
                          int32_t on_device);

/* One implicit Euler step from state xn by Newton's method, x in: the initial iterate, out: the
 * solution ([n][b], host or device per on_device).  F(x) = ||W R(x)||_2.  Each iteration assembles
 * J and S_e at x on the device, sets up the context's preconditioner on them (cptr_setup with the
 * model's weights) and solves J dx = -R to rtol_lin (cptr_solve); then a backtracking line search:
 * a = 1, 1/2, ... (at most 10 halvings) until F(x + a dx) <= (1 - 1e-4 a) F(x).  Converged when
 * F <= 1e-8 F(x^0), or when ||a dx|| <= 1e-8 ||x|| with F not above F(x^0).  Returns CPTR_OK,
 * CPTR_NOT_CONVERGED after max_newton iterations, or the errors of cptr_setup / cptr_solve. */
cptr_status cptr_newton(cptr_ctx *ctx, double *x, const double *xn, double rtol_lin, int32_t max_newton,
                        cptr_newton_stats *st, int32_t on_device);

#ifdef __cplusplus
}
#endif
#endif /* CPTR_H */
