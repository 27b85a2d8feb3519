// Shared declarations of the CPTR CUDA library (sm_103a).  Device data structures, error
// plumbing and the host-side launchers that the translation units share.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/cptr.h"

namespace cptr {

constexpr int kMaxLevels = 32;
constexpr int kMaxRestart = 32;
constexpr int kRedBlocks = 304;   // 2 x 152 SMs: fixed grid of the Krylov reductions
constexpr int kRedThreads = 256;

struct Error {
    cptr_status code;
    std::string msg;
};

// throw-free error propagation inside the library: every helper returns cptr_status and leaves
// its message in the context
#define CPTR_CUDA_TRY(ctx, call)                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return (ctx)->fail(CPTR_ECUDA, std::string(#call) + ": " +      \
                                                  cudaGetErrorString(e_));                     \
    } while (0)

#define CPTR_TRY(call)                                                                         \
    do {                                                                                       \
        cptr_status s_ = (call);                                                               \
        if (s_ != CPTR_OK) return s_;                                                          \
    } while (0)

// Device CSR matrix (int32 indices, FP64 values)
struct Csr {
    int32_t n = 0, nnz = 0;
    int32_t *rp = nullptr, *ci = nullptr;
    double *v = nullptr;
};

typedef __nv_bfloat16 bf16;

// launch shape of a row-parallel sparse kernel: G lanes per row (0: chosen from the average row
// length), T threads per block; picked per operator by the autotuner (amg_autotune, sell_autotune)
struct Shape {
    int16_t G = 0;
    int16_t T = 256;
};
enum { ST_F64 = 0, ST_F32 = 1, ST_BF16 = 2 };   // storage of matrix values

struct Level {
    Csr A;                 // level operator
    double *dinv = nullptr;// smoother D^{-1}
    Csr P, PT;             // interpolation and restriction (empty on the coarsest level)
    int32_t nc = 0;
    int32_t *cf = nullptr; // 1 = C, 2 = F
    double *b = nullptr, *x = nullptr, *t = nullptr, *r = nullptr;  // level work vectors
    // mixed-precision form: values of A, P, P^T stored in FP32 (levels 0, 1) or BF16 (levels
    // >= 2), D^{-1} and the work vectors in FP32
    int st = ST_F64;
    Shape sh_A, sh_PT, sh_P;   // launch shapes of the smoother/residual, restriction, prolongation
    void *Av_lo = nullptr, *Pv_lo = nullptr, *PTv_lo = nullptr;
    float *dinv32 = nullptr;
    float *b32 = nullptr, *x32 = nullptr, *t32 = nullptr, *r32 = nullptr;
    // unknown-based AMG (Sec. 3.4): the unknown of every row (0 pressure, 1 temperature; null for
    // classical AMG) and the number of pressure rows, which come first
    int32_t *fn = nullptr;
    int32_t np = 0;
};

// a level as the fused coarse-level kernels see it (device array, one per hierarchy and cycle
// precision): operators with their value storage, smoother diagonal and work vectors
struct LevelDev {
    int32_t n, st;
    const int32_t *rp, *ci, *Prp, *Pci, *PTrp, *PTci;
    const void *v, *Pv, *PTv, *dinv;
    void *b, *x, *t, *r;
};

struct Hier {
    int nlev = 0;
    Level L[kMaxLevels];
    double *cinv = nullptr;  // coarsest level: dense inverse (row-major), if dense
    int dense = 0;
    double op_complexity = 0.0;
    int fuse_l0 = -1;                 // levels fuse_l0 .. nlev-2 run in the fused coarse kernels
    LevelDev *ldev64 = nullptr, *ldev32 = nullptr;   // device descriptors (FP64 / mixed cycle)
    // the coarsest inverse runs on the context's coarse stream while the set-up goes on
    int32_t *gj_flag = nullptr;       // singular coarsest matrix
    cudaEvent_t gj_done = nullptr;    // recorded on the coarse stream after the inverse
    bool gj_pending = false;
};

// Arnoldi/Givens state kept on the device (one per context)
struct KState {
    int32_t k, done, breakdown, wait_err;  // columns completed in this cycle, flags; a bounded
                                           // device-side wait gave up (ILU sweeps)
    uint32_t ticket;                  // last-block ticket of the reductions
    int32_t active;                   // ensemble: this instance iterates in the current cycle
    int32_t its;                      // ensemble: Arnoldi steps this instance has taken
    int32_t pad3;
    double bnorm, beta, tol_abs, hnorm, est, true_res;
    double h[kMaxRestart + 1];       // first-pass CGS coefficients
    double h2[kMaxRestart + 1];      // second-pass CGS coefficients
    double g[kMaxRestart + 1], cs[kMaxRestart], sn[kMaxRestart], y[kMaxRestart];
    double H[(kMaxRestart + 1) * kMaxRestart];  // column-major, H[col * (m+1) + row]
};

// the leading fields of a KState (the part the host polls)
struct KHdr {
    int32_t k, done, breakdown, wait_err;
    uint32_t ticket;
    int32_t active, its, pad3;
    double bnorm, beta, tol_abs, hnorm, est, true_res;
};
static_assert(sizeof(KHdr) == offsetof(KState, h), "KHdr mirrors the head of KState");

struct Ctx;

// ---- launch counting and event timing of kernel families -----------------------------------------
void note_launch();          // every kernel launch of the library calls this once
void note_launches(int64_t n);  // a graph replay of n kernel nodes
int64_t launch_count();
void begin_capture_count();  // launches noted on this thread while capturing are not counted...
int64_t end_capture_count(); // ...but returned here (the graph's kernel node count)
// families 0-6 are switched on by bits 0-6 of the profiling mask; bit 7 switches on the eight
// fine-level V-cycle kernels PF_VC + 4 * hierarchy (0 pressure or p-T, 1 temperature) + step
// (0 pre-smoothing + residual, 1 restriction, 2 prolongation, 3 post-smoothing)
enum { PF_SPMV = 0, PF_STAGE1 = 1, PF_RESID = 2, PF_ILU = 3, PF_ARNOLDI = 4, PF_ILU_FWD = 5, PF_ILU_BWD = 6,
       PF_FAMILIES = 8, PF_VC = 8, PF_N = 16 };
constexpr int kSetupPhases = 8;
struct Prof {
    uint32_t mask = 0;
    std::vector<cudaEvent_t> ev;   // pairs (begin, end)
    std::vector<int> fam;
    size_t used = 0;               // slots recorded by direct launches since the last collect
    bool capturing = false;
    std::vector<size_t> gslots;    // slots recorded inside the captured iteration graph
    double ms[PF_N] = {0};
    int64_t cnt[PF_N] = {0};
    double setup_ms[kSetupPhases] = {0};   // set-up phases (host clock, after a stream sync): see SETUP_*
};
// set-up phases: inputs + decoupling + extraction; AMG coarsening (strength + PMIS + interp);
// AMG Galerkin products (transpose + two SpGEMMs); AMG coarsest inverse; ILU host work (ordering,
// level sets, sweep tables); ILU factorisation; SELL layout + mixed-precision copies; other
enum { SETUP_INPUTS = 0, SETUP_COARSEN = 1, SETUP_RAP = 2, SETUP_COARSEST = 3, SETUP_ILU_HOST = 4,
       SETUP_ILU_FACTOR = 5, SETUP_LAYOUT = 6, SETUP_OTHER = 7 };
// adds the host time since *t0 (after syncing the context's stream) to set-up phase `phase`
void setup_tick(Ctx *c, int phase, double *t0);
double host_ms();
int prof_begin(const Ctx *c, int fam);
void prof_end(const Ctx *c, int slot);
void prof_reset(Ctx *c);
cptr_status prof_collect(Ctx *c);
cptr_status prof_collect_graph(Ctx *c);
void prof_begin_capture(Ctx *c);
void prof_end_capture(Ctx *c);
cptr_status build_iteration_graph(Ctx *c);

// ---- memory helpers ----------------------------------------------------------------------------
// Device memory comes from a stream-ordered pool owned by the context (freed memory stays in
// the pool for the next set-up).  dfree releases on the stream of the context whose API call is
// running on this thread (CtxScope), or synchronously when none is.
cptr_status dalloc(Ctx *c, void **p, size_t bytes);
cptr_status copy_to_host(Ctx *c, void *dst, const void *src, size_t bytes);
cptr_status host_pattern(Ctx *c);   // h_ci and h_diag from the device pattern, once per set-up
struct CtxScope {
    explicit CtxScope(Ctx *c);
    ~CtxScope();
    Ctx *prev;
};
template <typename T>
inline cptr_status dalloc_t(Ctx *c, T **p, size_t count) {
    return dalloc(c, reinterpret_cast<void **>(p), count * sizeof(T));
}
void dfree(void *p);
void csr_free(Csr &a);

// ---- sparse.cu ---------------------------------------------------------------------------------
cptr_status scan_exclusive(Ctx *c, const int32_t *in, int32_t *out, int32_t n, int32_t *total_host);
void launch_decouple(const Ctx *c, const double *Araw, const double *W, double *A);
void launch_weight_vec(const Ctx *c, const double *W, const double *rhs, double *out);
void launch_extract(const Ctx *c, int u, int w, double *out);   // field (u, w) of A' (of G A' if decoupled)
cptr_status decoupling_setup(Ctx *c);                            // D_i of QI / TI into c->Ddec
void launch_check_finite(const Ctx *c, const double *v, int64_t n, int32_t *flag);
cptr_status sell_build(Ctx *c);
void launch_bsr_to_sell(const Ctx *c);
void launch_bsr_spmv(const Ctx *c, const double *x, double *y);
void launch_bsr_resid(const Ctx *c, const double *x, const double *v, double *y);
void launch_bsr_resid_pt(const Ctx *c, const double *dp, const double *dT, const double *v, double *b1);
// ts, to (optional): also to = ts * y per row (the first smoothing step of a V-cycle on y)
void launch_csr_spmv(cudaStream_t s, const Csr &A, const double *x, double *y, double alpha, const double *c0,
                     const double *ts = nullptr, double *to = nullptr);
// y = A x (mode 0), y = c0 - A x (mode 1), y += A x (mode 2); values VT, vectors and sums XT
template <typename VT, typename XT>
void launch_csr_spmv_t(cudaStream_t s, int32_t n, int32_t nnz, const int32_t *rp, const int32_t *ci, const VT *v,
                       const XT *x, XT *y, int mode, const XT *c0, Shape sh = Shape(), int32_t ncol = INT32_MAX,
                       const XT *ts = nullptr, XT *to = nullptr);
cptr_status to_lower(Ctx *c, const double *src, int64_t n, int st, void **dst);
void launch_d2f(const Ctx *c, const double *a, float *b, int64_t n);
void launch_f2d(const Ctx *c, const float *a, double *b, int64_t n);
// bp, bT of stage 1 from v (decoupled when the context has D); sp/tp, sT/tT (optional): also
// tp = sp * bp, tT = sT * bT (the first smoothing step of a V-cycle on bp or bT)
template <typename XT>
void launch_gather_pt(const Ctx *c, const double *v, XT *bp, XT *bT, const XT *sp = nullptr, XT *tp = nullptr,
                      const XT *sT = nullptr, XT *tT = nullptr);
template <typename XT> void launch_scatter_pt(const Ctx *c, const XT *dp, const XT *dT, double *x1);
void launch_resid_pt32(const Ctx *c, const float *dp, const float *dT, const double *v, float *b1);
void launch_sub(cudaStream_t s, int32_t n, const double *a, const double *b, double *out);

// the stage-1 kinds that build the S~_T hierarchy (the unknown-based AMG keeps its A_00 hierarchy
// in the pressure slot)
inline bool uses_T(int s1) { return s1 != CPTR_STAGE1_NONE && s1 != CPTR_STAGE1_CPR && s1 != CPTR_STAGE1_UAMG; }

// ---- amg.cu ------------------------------------------------------------------------------------
cptr_status build_a00(Ctx *c, Csr &A00, int32_t **fn);   // A_00 in unknown-wise order, unknown ids
cptr_status schur_diag(Ctx *c, Csr &S);                  // S~_diag = A_TT - A_Tp diag(A_pp)^{-1} A_pT
cptr_status amg_autotune(Ctx *c, Hier &h);    // launch shapes of every level's kernels
cptr_status amg_fuse_setup(Ctx *c, Hier &h);  // descriptors of the fused coarse levels
cptr_status sell_autotune(Ctx *c);           // threads per block of the SELL SpMV
cptr_status ilu_autotune(Ctx *c);            // grid and poll back-off of the ILU(0) sweeps
cptr_status amg_setup(Ctx *c, Hier &h, const int32_t *rp, const int32_t *ci, const double *v, int32_t n,
                      const int32_t *fn0 = nullptr, int32_t np0 = 0);
void amg_free(Hier &h);
// Loads the kernels a set-up may first launch while other work of the set-up is running (the
// cooperative coarsest inverse): with lazy module loading, a first load during the set-up stalled
// its other thread for ~0.4 s on a 2M-cell system.
void amg_preload();
cptr_status amg_coarsest_wait(Ctx *c, Hier &h);   // join the coarse stream's inverse; its status
// x = one V(1,1)-cycle on b; t_ready: the finest level's t = D^{-1} b was written by b's producer
void amg_vcycle(const Ctx *c, const Hier &h, const double *b, double *x, bool t_ready = false);
void amg_vcycle32(const Ctx *c, const Hier &h, const float *b, float *x, bool t_ready = false);
cptr_status amg_lower_precision(Ctx *c, Hier &h);

// ---- ilu.cu ------------------------------------------------------------------------------------
cptr_status ilu_setup(Ctx *c);
void ilu_free(Ctx *c);
void ilu_sym_free(Ctx *c);                               // the pattern-only tables kept across set-ups
void ilu_apply(const Ctx *c, const double *r, double *z, const double *dp, const double *dT);
void ilu_apply_into(const Ctx *c, const double *r, double *z, double *ybuf, double *zbuf);
void ilu_apply32(const Ctx *c, const float *r, double *z, const float *dp, const float *dT);

// ---- ilu_tile.cu -------------------------------------------------------------------------------
bool tile_grid(Ctx *c);                                  // detect the box; sets c->tl_dims
void tile_candidates(const Ctx *c, int k, std::vector<std::pair<int, int>> &out);   // best k tile shapes
cptr_status tile_setup(Ctx *c, int Ty, int Tz);          // tables of both sweeps; sets c->tl_ok
void tile_free(Ctx *c);
template <typename T, typename RT, typename XT>
void tile_apply(const Ctx *c, const RT *r, double *z, const XT *dp, const XT *dT);   // both sweeps (after the fill)

// ---- model.cu ----------------------------------------------------------------------------------
void model_free(Ctx *c);

// ---- krylov.cu ---------------------------------------------------------------------------------
cptr_status fgmres_solve(Ctx *c, const double *bw, double *x, double rtol, cptr_stats *st);
// ensemble (one block-diagonal set-up, FGMRES per instance): x and bw are union vectors
cptr_status fgmres_solve_batch(Ctx *c, const double *bw, double *x, double rtol, cptr_stats *st);
void free_batch(Ctx *c);
// learned Schur scaling (learned.cu)
cptr_status learned_prepare(Ctx *c);                       // saturation terms (needs c->A)
cptr_status learned_schur(Ctx *c, bool *used);             // S~_T = diag(s) S~_T into c->St
cptr_status learned_features(Ctx *c, double *feat);       // [n][16] device
cptr_status mlp_loss_grad(Ctx *c, const double *feat, const double *target, int32_t n, const float *params,
                          float *grad, double *loss);      // device arrays
cptr_status mlp_train(Ctx *c, const double *feat, const double *target, int32_t n, float *params, int32_t steps,
                      float lr, double *loss_hist);        // device arrays, loss_hist host
cptr_status mlp_infer(Ctx *c, const double *feat, int32_t n, float *y);   // device arrays
void apply_stage1(const Ctx *c, const double *v, const double **dp, const double **dT);
void apply_stage1_32(const Ctx *c, const double *v, const float **dp, const float **dT);
void apply_precond(const Ctx *c, const double *v, double *z);

// tables of one chunked ILU(0) sweep (see ilu.cu)
struct CwTables {
    int32_t nchunks = 0, D = 0, W = 1, maxw = 0, threads = 0, smem = 0, ns = 2, maxlev = 0;
    int32_t *clev = nullptr, *lptr = nullptr, *prow = nullptr, *code = nullptr;
    int32_t *started = nullptr;   // per chunk: it has finished its first levels (reset per sweep)
    void *val = nullptr;   // factor blocks (and inverted pivot blocks), FP64 or FP32
};

// tables of one tiled ILU(0) sweep (see ilu_tile.cu): tiles in processing order, their level
// pointers, and one record per position (row, dependency codes, factor blocks)
struct TileTables {
    int32_t ntiles = 0, nlev = 0, D = 0, MW = 0, RS = 0, R = 0, P = 2, smem = 0, threads = 0, grid = 0, maxnl = 0;
    int32_t *tlev = nullptr, *lptr = nullptr;
    unsigned char *rec = nullptr;
};

// Pattern-only ILU tables kept from one set-up to the next while the caller's block pattern and the
// ILU options that shape them are unchanged (the pattern is compared on the device at every set-up):
// the level sets of both sweeps, and the grid dimensions and tile structure of the tiled sweeps.
// Values (factors, packed records) are always rebuilt.
struct IluSym {
    int32_t n = -1, b = 0, nnzb = 0, order = -1, fill = -1;
    int32_t *rp = nullptr, *ci = nullptr;        // the pattern the tables belong to (device copy)
    bool current = false;                        // matched or rebuilt by this set-up's ilu_setup
    bool lv = false;                             // level sets held
    int32_t *lvl[2] = {}, *inv[2] = {}, *levr[2] = {};   // forward, backward
    std::vector<int32_t> lptr[2];
    int grid = -1;                               // tiled-sweep grid found (1), not found (0), unknown (-1)
    int32_t dims[3] = {0, 0, 0};
    int tile_ty = 0, tile_tz = 0, tile_prec = -1;  // tile structure held for this shape and precision
    TileTables tt[2];                            // its sizes, with tlev and lptr owned here (rec unused)
    int32_t *hdr[2] = {}, *kidx[2] = {};
    size_t tlev_n[2] = {}, lptr_n[2] = {};
    // the structure of the grouped-level tables of both sweeps for one group size (grp): entry
    // counts and offsets per position, dependency positions and right-hand-side sources, and the
    // SELL layout (chunk offsets, slot columns, slot -> entry index) of the M and W tables
    struct GroupDir {
        int32_t *mcnt = nullptr, *ccnt = nullptr, *moff = nullptr, *coff = nullptr, *mdep = nullptr, *cdep = nullptr;
        int32_t mtot = 0, ctot = 0;
        int64_t *off[2] = {};
        int32_t *col[2] = {}, *kidx[2] = {};
        int64_t ns[2] = {};
    };
    int grp = 0;
    GroupDir gd[2];
};

// ---- the context -------------------------------------------------------------------------------
struct Ctx {
    cptr_options o{};
    cudaStream_t stream = nullptr;
    cudaMemPool_t pool = nullptr;
    std::string err;
    bool ready = false;
    int32_t n = 0, b = 0, ps = 0, ts = 1, nnzb = 0;
    // pattern (device) and its host copy
    int32_t *rp = nullptr, *ci = nullptr, *diag = nullptr;
    std::vector<int32_t> h_rp, h_ci, h_diag;
    double *A = nullptr;     // decoupled A' (BSR, row-major blocks; set-up only)
    int32_t sell_nch = 0;    // A' for the solve: SELL-32 block layout (see sparse.cu)
    int64_t *sell_off = nullptr;
    int32_t *sell_col = nullptr;
    double *sell_val = nullptr;
    int64_t sell_bytes = 0, sell_nvals = 0;
    Shape sell_shape;        // threads per block of the SELL kernels (G unused)
    std::map<uint64_t, Shape> tune_cache;   // autotuned shapes by (kernel, size, storage)
    double *W = nullptr;     // per-cell weights (n * b * b)
    double *App = nullptr, *ApT = nullptr, *ATp = nullptr, *St = nullptr;  // cell-pattern fields
    // learned Schur scaling: the base approximation once St holds the scaled one, the per-cell
    // saturation terms of features 7 and 8, the row scaling of the last set-up, the network (FP32)
    double *lf_base = nullptr, *lf_sat = nullptr, *lf_s = nullptr;
    float *mlp = nullptr;
    int32_t schur_used = 0;
    Hier hp, hT;
    // ILU(0): factors in the pattern of the factorised matrix (A' in the caller's cell order, or
    // with cells permuted by colour), diagonal slots hold inverted pivot blocks
    double *LU = nullptr;
    int32_t *ilu_rp = nullptr, *ilu_ci = nullptr, *ilu_diag = nullptr;
    bool ilu_owns_pattern = false;   // false: the ILU pattern aliases rp/ci/diag
    int32_t *ilu_rowmap = nullptr;     // multicolour: row of the factorised matrix -> original row
    int32_t *ilu_flags = nullptr;      // per-row "factored" flags of the one-launch factorisation
    int32_t ilu_flags_n = 0, ilu_epoch = 0;
    IluSym isym;                                       // pattern-only ILU tables of the last set-up
    int32_t *part = nullptr, n_part = 0;               // cell partition of a block-Jacobi ILU (device)
    int32_t nlev_f = 0, nlev_b = 0;
    int32_t *lvl_f = nullptr, *lvl_b = nullptr;       // rows sorted by level (device)
    std::vector<int32_t> h_lptr_f, h_lptr_b;           // level pointers (host)
    double *ybuf = nullptr, *zbuf = nullptr;           // ILU intermediate vectors
    // ILU(0) solves, one launch per sweep: rows in level order, factors in SELL-32 chunks
    int32_t *sf_pos_f = nullptr, *sf_pos_b = nullptr;  // level-ordered position -> row
    int32_t *sf_bmap = nullptr;                        // backward position -> forward position
    int64_t *sf_off_f = nullptr, *sf_off_b = nullptr;  // chunk slot offsets
    int32_t *sf_col_f = nullptr, *sf_col_b = nullptr;  // dependency positions (-1 = padding)
    void *sf_val_f = nullptr, *sf_val_b = nullptr;     // L and U blocks (FP64, or FP32 when mixed)
    void *sf_dinv = nullptr;                           // inverted pivot blocks, backward order
    unsigned *sf_ticket = nullptr;                     // block tickets of the two sweeps
    void *sf_y = nullptr, *sf_z = nullptr;             // level-ordered y and z (sentinel-filled)
    CwTables cw_f, cw_b;                               // chunked wavefront sweeps (natural order)
    bool cw_ok = false, cw_use = false;                // built / chosen (autotuner may switch)
    // paired-level sweeps: a row of odd level substitutes its dependencies of the level
    // before, so that two levels run as one; main tables (off/col/val) and the tables of the part
    // that needs no other row's result (coff/ccol/cval)
    int64_t *sp_off_f = nullptr, *sp_off_b = nullptr, *sp_coff_f = nullptr, *sp_coff_b = nullptr;
    int32_t *sp_col_f = nullptr, *sp_col_b = nullptr, *sp_ccol_f = nullptr, *sp_ccol_b = nullptr;
    void *sp_val_f = nullptr, *sp_val_b = nullptr, *sp_cval_f = nullptr, *sp_cval_b = nullptr;   // FP64, or FP32 when mixed
    bool sp_ok = false, sp_use = false;                // built / chosen
    int sp_group = 0;                                  // levels per group of the tables built
    int sf_half = 1;                                   // grouped-level sweeps: lanes per row / 4 (1, 2 or 4)
    int32_t *sp_inv_f = nullptr, *sp_inv_b = nullptr;  // position of each row in either sweep
    int32_t *sp_levr_f = nullptr, *sp_levr_b = nullptr;   // level of each row in either sweep
    // tiled sweeps: a block owns a tile of grid lines and walks its own levels (natural order on
    // a Cartesian box, detected from the pattern)
    TileTables tl_f, tl_b;
    bool tl_ok = false, tl_use = false;                // built / chosen
    int32_t tl_dims[3] = {0, 0, 0};                    // detected nx, ny, nz (0: no box)
    int32_t tl_ty = 0, tl_tz = 0;                      // tile shape of the tables built
    int32_t tl_best_ty = 0, tl_best_tz = 0;            // tile shape the set-up chose (tuned or given)
    int32_t sf_grid = 4 * 152;                         // persistent grid of the sweeps (autotuned)
    int32_t sf_sleep = 20;                             // back-off between polls, ns (autotuned)
    int32_t inject_wait = 0;                           // failure injection (see cptr_inject_wait_timeout)
    double *never = nullptr;                           // a word no thread writes
    // preconditioner work
    double *bp = nullptr, *bT = nullptr, *xp = nullptr, *dp = nullptr, *dT = nullptr, *t1 = nullptr;
    double *b00 = nullptr, *x00 = nullptr;             // unknown-based AMG: [b_p; b_T], [d_p; d_T]
    double *Ddec = nullptr;                            // decoupling: D_i per cell, [n][2][b] (rows p, T)
    void *model = nullptr;                             // the finite-volume model of the Newton loop (model.cu)
    float *b0032 = nullptr, *x0032 = nullptr;
    double *b1 = nullptr;
    // mixed-precision form: FP32 copies of the stage-1 operators and the stage-1 vectors
    float *ApT32 = nullptr, *ATp32 = nullptr, *sell_val32 = nullptr;
    float *bp32 = nullptr, *bT32 = nullptr, *xp32 = nullptr, *dp32 = nullptr, *dT32 = nullptr, *t132 = nullptr;
    float *b132 = nullptr;
    // Krylov
    double *V = nullptr, *Z = nullptr, *w = nullptr, *bw = nullptr, *xw = nullptr, *partial = nullptr;
    double *vcur = nullptr, *zcur = nullptr;           // fixed in/out vectors of the captured step
    cudaStream_t cap_stream = nullptr;
    cudaStream_t side_stream = nullptr;   // set-up work that overlaps the main stream
    cudaStream_t coarse_stream = nullptr; // the coarsest AMG inverses, overlapping the rest of the set-up
    cudaStream_t amg_stream[2] = {};      // the hierarchies, each built by a host thread of its own
    cudaEvent_t amg_fork[2] = {};
    cudaEvent_t side_fork = nullptr, side_join = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaGraphExec_t cycle_exec = nullptr;   // a whole restart cycle: WHILE node over the Arnoldi step
    int64_t cycle_step_launches = 0;        // kernels per step of the cycle graph
    bool cycle_failed = false;              // not available here: per-step graphs are used
    int64_t graph_launches = 0;
    uint32_t graph_mask = 0;
    int32_t graph_inject = 0;
    KState *ks = nullptr;    // device
    KState *ks_host = nullptr;  // pinned mirror
    // ensemble: instances are consecutive cell ranges of the set-up system (block diagonal)
    int32_t n_inst = 0;
    std::vector<int32_t> inst_cell0;       // first cell of each instance, and n at the end
    int32_t n_tiles = 0;                   // union vector tiles, none straddles two instances
    int32_t *tile_inst = nullptr;          // tile -> instance
    int64_t *tile_beg = nullptr;           // tile -> [beg, end) in the union vector
    int32_t *inst_tile0 = nullptr;         // instance -> first tile (n_inst + 1 entries)
    KState *ksb = nullptr;                 // per-instance Krylov state (device)
    KHdr *hdr = nullptr, *hdr_host = nullptr;     // per-instance headers (+ the ILU wait flag)
    double *partial_b = nullptr;           // per-tile reduction partials
    cudaGraphExec_t bgraph_exec = nullptr;
    int64_t bgraph_launches = 0;
    cudaGraphExec_t bcycle_exec = nullptr;   // the ensemble's restart cycle as one graph launch
    int64_t bcycle_step_launches = 0;
    bool bcycle_failed = false;
    int32_t *flag = nullptr;    // device scratch flag
    int32_t *scan_tmp = nullptr; int64_t scan_tmp_len = 0;
    double setup_ms = 0.0;
    mutable Prof prof;

    cptr_status fail(cptr_status code, const std::string &m) {
        err = m;
        return code;
    }
};

// acc + sum over k0 <= k < k1 of v_k * x(col_k), added in k order (one fma per entry, the order
// of a plain row loop) by one thread.  The entries are taken U at a time: the U column indices and
// values are loaded first, then the U gathered x values, so a thread has U independent loads in
// flight instead of a chain of dependent ones per entry.
template <int U, typename XT, typename LV, typename LX>
__device__ __forceinline__ XT row_dot_batched(int32_t k0, int32_t k1, const int32_t *__restrict__ ci, LV ldv, LX ldx,
                                              XT acc) {
    for (int32_t k = k0; k < k1; k += U) {
        int32_t j[U];
        XT a[U], xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (k + u < k1) {
                j[u] = __ldg(ci + k + u);
                a[u] = ldv(k + u);
            }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (k + u < k1) xv[u] = ldx(j[u]);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (k + u < k1) acc = fma(a[u], xv[u], acc);
    }
    return acc;
}

// Index checks of the bounds-checking build (compiled with -DCPTR_CHECK into libcptr_check.so).
// chk(i, n, site) returns i when 0 <= i < n.  Otherwise it records the first failure of the
// translation unit (site, index, bound) and returns 0, so that the access stays inside the array and
// the kernel completes; every entry point then reports CPTR_ECHECK.  No trap and no device assert:
// the context stays usable.  In the normal build chk() is the identity.  Each translation unit
// keeps its own record (device symbols are per unit without relocatable device code) and registers
// host functions that read and clear it.
struct CheckRec {
    int32_t count, site;
    int64_t index, bound;
};
#ifdef CPTR_CHECK
void check_register(cudaError_t (*fetch)(CheckRec *), cudaError_t (*clear)());
struct CheckRegistration {
    CheckRegistration(cudaError_t (*fetch)(CheckRec *), cudaError_t (*clear)()) { check_register(fetch, clear); }
};
static __device__ CheckRec g_check_tu;
static cudaError_t check_fetch_tu(CheckRec *out) { return cudaMemcpyFromSymbol(out, g_check_tu, sizeof(CheckRec)); }
static cudaError_t check_clear_tu() {
    const CheckRec z{};
    return cudaMemcpyToSymbol(g_check_tu, &z, sizeof(CheckRec));
}
static CheckRegistration check_registration_tu(check_fetch_tu, check_clear_tu);
__device__ __forceinline__ int64_t chk(int64_t i, int64_t n, int site) {
    if (i >= 0 && i < n) return i;
    if (atomicAdd(&g_check_tu.count, 1) == 0) {
        g_check_tu.site = site;
        g_check_tu.index = i;
        g_check_tu.bound = n;
    }
    return 0;
}
#else
__device__ __forceinline__ int64_t chk(int64_t i, int64_t, int) { return i; }
#endif
// the sites of chk() (reported by number)
enum { CHK_SELL_COL = 1, CHK_CSR_COL = 2, CHK_VC_COL = 3, CHK_ILU_DEP = 4, CHK_ILU_PAIR = 5, CHK_FACTOR_COL = 6,
       CHK_FACTOR_DEP = 7, CHK_GATHER = 8 };
// a dependency position of the sweep tables: -1 marks an empty slot, anything else is checked
__device__ __forceinline__ int32_t chk_dep(int32_t c, int32_t n) {
    return c < 0 ? -1 : (int32_t)chk(c, n, CHK_ILU_DEP);
}
// true (and the context's error set) if a check of this process failed since the last call
cptr_status check_report(Ctx *c);

// Programmatic dependent launch: a kernel launched by launch_pdl may be scheduled while the kernel
// before it on the stream is still running, which hides the launch latency of short kernels in a
// chain (the V-cycle's).  Such a kernel calls pdl_wait() before its first global memory access:
// that waits until the previous kernel has completed and its writes are visible, then lets the
// next kernel on the stream be scheduled.  In a kernel launched without the attribute both
// instructions do nothing.
__device__ __forceinline__ void pdl_wait() {
    asm volatile("griddepcontrol.wait;\n\tgriddepcontrol.launch_dependents;" ::: "memory");
}
void note_launch();
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
    note_launch();
}

// lanes per row for a CSR kernel without a tuned shape: one lane per row on large operators with
// short rows (what the autotuner picks there on GB300: a cross-lane sum costs a warp-wide FP64
// instruction per step), otherwise from the average row length
inline int lanes_for(int32_t n, int32_t nnz) {
    double avg = n > 0 ? double(nnz) / n : 1.0;
    if (n >= 16384 && avg <= 24.0) return 1;
    if (avg <= 4.5) return 4;
    if (avg <= 9.0) return 8;
    if (avg <= 24.0) return 16;
    return 32;
}

}  // namespace cptr

// the opaque handle of the C ABI
struct cptr_ctx {
    cptr::Ctx c;
};
