// Right-preconditioned flexible GMRES(m) (Sec. 3 and Sec. 4: right-preconditioned GMRES,
// relative residual tolerance) with classical Gram-Schmidt and one full re-orthogonalisation
// (CGS2).  Each Gram-Schmidt pass is one streaming kernel that updates w and forms all partial
// dot products of the pass with warp-shuffle and block reductions; the last block to finish
// reduces the per-block partials in block order (deterministic) and, after the second pass,
// applies the Givens rotations on the device.  The two-stage preconditioner is driven from here.
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>

#include "common.cuh"

namespace cptr {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

enum { PASS_DOT = 0, PASS_UPD_DOT = 1, PASS_UPD_NORM = 2, PASS_NORM = 3 };
enum { FIN_H = 0, FIN_H2 = 1, FIN_GIVENS = 2, FIN_BNORM = 3, FIN_RESTART = 4, FIN_TRUE = 5 };

constexpr int kMaxC = kMaxRestart;   // columns per pass
constexpr int kPStride = kMaxC + 1;  // partial row stride

// the work of the last block of a reduction: res[] holds the reduced sums of the pass
__device__ void cgs_finish(KState *ks, const double *res, int fin, int j, int m, double rtol, int nc) {
    if (fin == FIN_H) {
        for (int q = 0; q < nc; ++q) ks->h[q] = res[q];
    } else if (fin == FIN_H2) {
        for (int q = 0; q < nc; ++q) ks->h2[q] = res[q];
    } else if (fin == FIN_GIVENS) {
        double hn = sqrt(res[0]);
        double *col = ks->H + (int64_t)j * (m + 1);
        for (int q = 0; q <= j; ++q) col[q] = ks->h[q] + ks->h2[q];
        col[j + 1] = hn;
        for (int q = 0; q < j; ++q) {
            double a = col[q], b = col[q + 1];
            col[q] = ks->cs[q] * a + ks->sn[q] * b;
            col[q + 1] = -ks->sn[q] * a + ks->cs[q] * b;
        }
        double a = col[j], b = col[j + 1];
        double den = sqrt(a * a + b * b);
        ks->cs[j] = a / den;
        ks->sn[j] = b / den;
        col[j] = den;
        col[j + 1] = 0.0;
        ks->g[j + 1] = -ks->sn[j] * ks->g[j];
        ks->g[j] = ks->cs[j] * ks->g[j];
        ks->hnorm = hn;
        ks->k = j + 1;
        ks->its += 1;
        ks->est = fabs(ks->g[j + 1]) / ks->bnorm;
        if (!isfinite(hn) || !isfinite(den) || !isfinite(ks->g[j])) { ks->breakdown = 1; ks->done = 1; }
        else if (fabs(ks->g[j + 1]) <= ks->tol_abs || hn == 0.0) ks->done = 1;
    } else if (fin == FIN_BNORM || fin == FIN_RESTART) {
        double beta = sqrt(res[0]);
        if (fin == FIN_BNORM) {
            ks->bnorm = beta;
            ks->tol_abs = rtol * beta;
        }
        ks->beta = beta;
        for (int q = 0; q <= m; ++q) ks->g[q] = 0.0;
        ks->g[0] = beta;
        ks->k = 0;
        ks->est = ks->bnorm > 0.0 ? beta / ks->bnorm : 0.0;
        if (!isfinite(beta)) { ks->breakdown = 1; ks->done = 1; }
        else ks->done = (beta <= ks->tol_abs) ? 1 : 0;
        ks->active = !ks->done;
    } else {  // FIN_TRUE
        ks->true_res = sqrt(res[0]);
    }
}

// The element loop of a Gram-Schmidt pass with NQ columns compiled in (NQ = nc rounded up to a
// multiple of 4, so at most 3 columns are carried as predicated-off work): each element reads w
// once, updates it (UPD) and adds its products to the per-column partial sums.
template <int PASS, int NQ>
__device__ __forceinline__ void cgs_elements(int64_t i0, int64_t i1, int64_t step, int64_t nb,
                                             const double *__restrict__ V, int nc, double *__restrict__ w,
                                             const double *scoef, double *acc) {
    constexpr bool UPD = PASS == PASS_UPD_DOT || PASS == PASS_UPD_NORM;
    constexpr bool NORM = PASS == PASS_UPD_NORM || PASS == PASS_NORM;
    for (int64_t i = i0; i < i1; i += step) {
        double wi = w[i];
        if (UPD) {
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nc) wi = fma(-scoef[q], __ldg(V + (int64_t)q * nb + i), wi);
            w[i] = wi;
        }
        if (NORM) {
            acc[0] = fma(wi, wi, acc[0]);
        } else {
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nc) acc[q] = fma(__ldg(V + (int64_t)q * nb + i), wi, acc[q]);
        }
    }
}

// Column sums over a warp: every lane holds P = 2^LP partial sums a[0..P); at each of LP halving
// steps a lane keeps half of its columns and adds its partner's values of them (so a step costs
// one FP64 add per kept column, not one per column), then the lanes sharing a column are added
// by a butterfly.  Lane l ends with the warp's sum of column l >> (5 - LP).  On GB300 a warp-wide
// FP64 add holds the FP64 pipe as long as an FMA, so this costs about P adds against 5 P for a
// shuffle tree per column.
template <int LP>
__device__ __forceinline__ double warp_colsum(double *a, int lane) {
    constexpr int P = 1 << LP;
#pragma unroll
    for (int st = 0; st < LP; ++st) {
        const int o = 16 >> st;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int q = 0; q < (P >> (st + 1)); ++q) {
            const int hf = P >> (st + 1);
            const double send = up ? a[q] : a[q + hf];
            const double keep = up ? a[q + hf] : a[q];
            a[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    double v = a[0];
#pragma unroll
    for (int o = 16 >> LP; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// A pass's element loop and its warp sums with NQ columns compiled in; red[wid][c] receives the
// warp's sum of column c (columns nc..P-1 carry zeros)
template <int PASS, int NQ>
__device__ __forceinline__ void cgs_pass(int64_t i0, int64_t i1, int64_t step, int64_t nb, const double *V, int nc,
                                         double *w, const double *scoef, double (*red)[kMaxC], int lane, int wid) {
    constexpr bool NORM = PASS == PASS_UPD_NORM || PASS == PASS_NORM;
    constexpr int LP = NORM ? 0 : (NQ <= 4 ? 2 : NQ <= 8 ? 3 : NQ <= 16 ? 4 : 5);
    constexpr int SH = 5 - LP;
    double acc[1 << LP];
#pragma unroll
    for (int q = 0; q < (1 << LP); ++q) acc[q] = 0.0;
    cgs_elements<PASS, NQ>(i0, i1, step, nb, V, nc, w, scoef, acc);
    const double v = warp_colsum<LP>(acc, lane);
    if ((lane & ((1 << SH) - 1)) == 0) red[wid][lane >> SH] = v;
}

// NQ = nc rounded up to a multiple of 4: the columns past nc are predicated off, and a
// predicated-off FP64 instruction still takes its turn on the pipe
template <int PASS>
__device__ __forceinline__ void cgs_dispatch(int64_t i0, int64_t i1, int64_t step, int64_t nb, const double *V, int nc,
                                             double *w, const double *scoef, double (*red)[kMaxC], int lane, int wid) {
    constexpr bool NORM = PASS == PASS_UPD_NORM || PASS == PASS_NORM;
    constexpr bool UPD = PASS == PASS_UPD_DOT || PASS == PASS_UPD_NORM;
    if (NORM && !UPD) {
        cgs_pass<PASS, 1>(i0, i1, step, nb, V, nc, w, scoef, red, lane, wid);
        return;
    }
    switch ((nc + 3) >> 2) {
    case 0:
    case 1: cgs_pass<PASS, 4>(i0, i1, step, nb, V, nc, w, scoef, red, lane, wid); break;
    case 2: cgs_pass<PASS, 8>(i0, i1, step, nb, V, nc, w, scoef, red, lane, wid); break;
    case 3: cgs_pass<PASS, 12>(i0, i1, step, nb, V, nc, w, scoef, red, lane, wid); break;
    case 4: cgs_pass<PASS, 16>(i0, i1, step, nb, V, nc, w, scoef, red, lane, wid); break;
    case 5: cgs_pass<PASS, 20>(i0, i1, step, nb, V, nc, w, scoef, red, lane, wid); break;
    case 6: cgs_pass<PASS, 24>(i0, i1, step, nb, V, nc, w, scoef, red, lane, wid); break;
    case 7: cgs_pass<PASS, 28>(i0, i1, step, nb, V, nc, w, scoef, red, lane, wid); break;
    default: cgs_pass<PASS, 32>(i0, i1, step, nb, V, nc, w, scoef, red, lane, wid); break;
    }
}

// One Gram-Schmidt pass over v_0..v_{nc-1} (columns of V, stride nb):
//   PASS_DOT       partial[q] = v_q . w
//   PASS_UPD_DOT   w -= sum_q coef_q v_q; partial[q] = v_q . w
//   PASS_UPD_NORM  w -= sum_q coef_q v_q; partial = w . w
//   PASS_NORM      partial = w . w
template <int PASS>
__global__ void __launch_bounds__(kRedThreads) k_cgs(int64_t nb, const double *__restrict__ V, int nc,
                                                    double *__restrict__ w, const double *__restrict__ coef,
                                                    double *__restrict__ partial, KState *ks, int fin, int j, int m,
                                                    double rtol, int jdev) {
    __shared__ double scoef[kMaxC];
    __shared__ double red[kRedThreads / 32][kMaxC];
    __shared__ bool last;
    if (ks->done && fin <= FIN_GIVENS) return;   // nothing after convergence in this cycle
    if (jdev) {                                   // column index from the device state (graphs)
        j = ks->k;
        nc = j + 1;
    }
    constexpr bool UPD = PASS == PASS_UPD_DOT || PASS == PASS_UPD_NORM;
    constexpr bool NORM = PASS == PASS_UPD_NORM || PASS == PASS_NORM;
    if (UPD && threadIdx.x < kMaxC) scoef[threadIdx.x] = threadIdx.x < nc ? coef[threadIdx.x] : 0.0;
    __syncthreads();
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int na = NORM ? 1 : nc;
    cgs_dispatch<PASS>((int64_t)blockIdx.x * blockDim.x + threadIdx.x, nb, stride, nb, V, nc, w, scoef, red, lane, wid);
    __syncthreads();
    if (threadIdx.x < na) {
        double s = 0.0;
        for (int w8 = 0; w8 < kRedThreads / 32; ++w8) s += red[w8][threadIdx.x];
        partial[(int64_t)blockIdx.x * kPStride + threadIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&ks->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    // last block: one warp per column; lane l sums blocks l, l+32, ... and the lanes are combined
    // by a fixed shuffle tree (the same order every run).  A lane loads its blocks' partials
    // before adding them, so a column costs one L2 round trip rather than one per block it sums.
    __threadfence();
    __shared__ double res[kMaxC];
    constexpr int kPU = (kRedBlocks + 31) / 32;   // partials per lane in one batch of loads
    for (int q = wid; q < na; q += kRedThreads / 32) {
        double s = 0.0;
        for (unsigned b0 = lane; b0 < gridDim.x; b0 += 32 * kPU) {
            double pv[kPU];
#pragma unroll
            for (int u = 0; u < kPU; ++u) {
                const unsigned bb = b0 + 32u * u;
                pv[u] = bb < gridDim.x ? __ldcg(partial + (int64_t)bb * kPStride + q) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < kPU; ++u)
                if (b0 + 32u * u < gridDim.x) s += pv[u];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) res[q] = s;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    ks->ticket = 0;
    cgs_finish(ks, res, fin, j, m, rtol, nc);
}

// dst = src / scale, scale = ks->hnorm (which = 0) or ks->beta (which = 1); skipped if 0 or done.
// jdev: dst is column ks->k of the block starting at dst (the column after the Givens update).
__global__ void k_scale(int64_t nb, const double *__restrict__ src, double *__restrict__ dst, const KState *ks,
                        int which, int check_done, int jdev) {
    if (check_done && ks->done) return;
    if (jdev) dst += (int64_t)ks->k * nb;
    double s = which == 0 ? ks->hnorm : ks->beta;
    if (!(s > 0.0)) return;
    double inv = 1.0 / s;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += stride) dst[i] = src[i] * inv;
}

// copy between a fixed vector and column ks->k of a column block: dir 0 vec = base[k],
// dir 1 base[k] = vec
__global__ void k_copy_col(int64_t nb, double *__restrict__ base, double *__restrict__ vec, const KState *ks,
                           int dir) {
    double *col = base + (int64_t)ks->k * nb;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += stride) {
        if (dir == 0) vec[i] = col[i];
        else col[i] = vec[i];
    }
}

// y = H^{-1} g (upper triangular, k x k)
__global__ void k_trisolve(KState *ks, int m) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int k = ks->k;
    for (int i = k - 1; i >= 0; --i) {
        double s = ks->g[i];
        for (int q = i + 1; q < k; ++q) s -= ks->H[(int64_t)q * (m + 1) + i] * ks->y[q];
        ks->y[i] = s / ks->H[(int64_t)i * (m + 1) + i];
    }
}

// x += sum_{q < k} y_q z_q
__global__ void __launch_bounds__(256) k_update_x(int64_t nb, const double *__restrict__ Z, const KState *ks,
                                                  double *__restrict__ x) {
    __shared__ double sy[kMaxC];
    int k = ks->k;
    if (threadIdx.x < kMaxC) sy[threadIdx.x] = threadIdx.x < k ? ks->y[threadIdx.x] : 0.0;
    __syncthreads();
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += stride) {
        double s = x[i];
#pragma unroll
        for (int q = 0; q < kMaxC; ++q)
            if (q < k) s = fma(sy[q], __ldg(Z + (int64_t)q * nb + i), s);
        x[i] = s;
    }
}

template <typename XT>
__global__ void k_add_x1(int32_t n, int b, int ps, int ts, const XT *dp, const XT *dT, const XT *b1, double *z) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int q = 0; q < b; ++q) {
        int64_t o = (int64_t)i * b + q;
        double add = 0.0;
        if (dp && q == ps) add = (double)dp[i];
        if (dT && q == ts) add = (double)dT[i];
        z[o] = (double)b1[o] + add;
    }
}

// ------------------------------------------------------------------------------------------------
// stage 1 (Sec. 3.1 CPR; Sec. 3.3 the block preconditioner and its variants)
void apply_stage1(const Ctx *c, const double *v, const double **pdp, const double **pdT) {
    cudaStream_t s = c->stream;
    Csr ATp{c->n, c->nnzb, c->rp, c->ci, c->ATp}, ApT{c->n, c->nnzb, c->rp, c->ci, c->ApT};
    *pdp = nullptr;
    *pdT = nullptr;
    int mode = c->o.stage1;
    if (mode == CPTR_STAGE1_NONE) return;
    // Every right-hand side of a V-cycle below is written together with its finest level's
    // t = D^{-1} b (the first smoothing step), so the V-cycles start from it (t_ready).
    const Level &P0 = c->hp.L[0], &T0 = c->hT.L[0];
    if (mode == CPTR_STAGE1_UAMG) {   // Sec. 3.4: one unknown-based V-cycle on A_00 [d_p; d_T] = [b_p; b_T]
        launch_gather_pt<double>(c, v, c->b00, c->b00 + c->n, P0.dinv, P0.t, P0.dinv + c->n, P0.t + c->n);
        amg_vcycle(c, c->hp, c->b00, c->x00, true);
        *pdp = c->x00;
        *pdT = c->x00 + c->n;
        return;
    }
    const bool t_direct = mode == CPTR_STAGE1_UPPER || mode == CPTR_STAGE1_BD;   // b_T itself goes to a V-cycle
    launch_gather_pt<double>(c, v, c->bp, c->bT, P0.dinv, P0.t, t_direct ? T0.dinv : nullptr,
                             t_direct ? T0.t : nullptr);
    switch (mode) {
    case CPTR_STAGE1_FULL:
        amg_vcycle(c, c->hp, c->bp, c->xp, true);                               // 1. A_pp x_p = b_p
        launch_csr_spmv(s, ATp, c->xp, c->t1, 1.0, c->bT, T0.dinv, T0.t);      // 2. b~_T = b_T - A_Tp x_p
        amg_vcycle(c, c->hT, c->t1, c->dT, true);                               // 3. S~_T d_T = b~_T
        launch_csr_spmv(s, ApT, c->dT, c->t1, 1.0, c->bp, P0.dinv, P0.t);      // 4. b~_p = b_p - A_pT d_T
        amg_vcycle(c, c->hp, c->t1, c->dp, true);                               // 5. A_pp d_p = b~_p
        break;
    case CPTR_STAGE1_LOWER:
        amg_vcycle(c, c->hp, c->bp, c->dp, true);
        launch_csr_spmv(s, ATp, c->dp, c->t1, 1.0, c->bT, T0.dinv, T0.t);
        amg_vcycle(c, c->hT, c->t1, c->dT, true);
        break;
    case CPTR_STAGE1_UPPER:
        amg_vcycle(c, c->hT, c->bT, c->dT, true);
        launch_csr_spmv(s, ApT, c->dT, c->t1, 1.0, c->bp, P0.dinv, P0.t);
        amg_vcycle(c, c->hp, c->t1, c->dp, true);
        break;
    case CPTR_STAGE1_BD:
        amg_vcycle(c, c->hp, c->bp, c->dp, true);
        amg_vcycle(c, c->hT, c->bT, c->dT, true);
        break;
    case CPTR_STAGE1_CPR:
        amg_vcycle(c, c->hp, c->bp, c->dp, true);
        *pdp = c->dp;
        return;
    }
    *pdp = c->dp;
    *pdT = c->dT;
}

// stage 1 of the mixed-precision form: the same steps in FP32 vectors with the FP32/BF16 hierarchy
void apply_stage1_32(const Ctx *c, const double *v, const float **pdp, const float **pdT) {
    cudaStream_t s = c->stream;
    const int32_t n = c->n, nnz = c->nnzb;
    // as in apply_stage1: every V-cycle right-hand side comes with its finest level's t = D^{-1} b
    const Level &P0 = c->hp.L[0], &T0 = c->hT.L[0];
    auto Tp = [&](const float *x, float *y, const float *c0) {   // y = c0 - A_Tp x, for the T V-cycle
        launch_csr_spmv_t<float, float>(s, n, nnz, c->rp, c->ci, c->ATp32, x, y, 1, c0, Shape(), n, T0.dinv32, T0.t32);
    };
    auto pT = [&](const float *x, float *y, const float *c0) {   // y = c0 - A_pT x, for the p V-cycle
        launch_csr_spmv_t<float, float>(s, n, nnz, c->rp, c->ci, c->ApT32, x, y, 1, c0, Shape(), n, P0.dinv32, P0.t32);
    };
    *pdp = nullptr;
    *pdT = nullptr;
    int mode = c->o.stage1;
    if (mode == CPTR_STAGE1_NONE) return;
    if (mode == CPTR_STAGE1_UAMG) {
        launch_gather_pt<float>(c, v, c->b0032, c->b0032 + n, P0.dinv32, P0.t32, P0.dinv32 + n, P0.t32 + n);
        amg_vcycle32(c, c->hp, c->b0032, c->x0032, true);
        *pdp = c->x0032;
        *pdT = c->x0032 + n;
        return;
    }
    const bool t_direct = mode == CPTR_STAGE1_UPPER || mode == CPTR_STAGE1_BD;   // b_T itself goes to a V-cycle
    launch_gather_pt<float>(c, v, c->bp32, c->bT32, P0.dinv32, P0.t32, t_direct ? T0.dinv32 : nullptr,
                            t_direct ? T0.t32 : nullptr);
    switch (mode) {
    case CPTR_STAGE1_FULL:
        amg_vcycle32(c, c->hp, c->bp32, c->xp32, true);
        Tp(c->xp32, c->t132, c->bT32);
        amg_vcycle32(c, c->hT, c->t132, c->dT32, true);
        pT(c->dT32, c->t132, c->bp32);
        amg_vcycle32(c, c->hp, c->t132, c->dp32, true);
        break;
    case CPTR_STAGE1_LOWER:
        amg_vcycle32(c, c->hp, c->bp32, c->dp32, true);
        Tp(c->dp32, c->t132, c->bT32);
        amg_vcycle32(c, c->hT, c->t132, c->dT32, true);
        break;
    case CPTR_STAGE1_UPPER:
        amg_vcycle32(c, c->hT, c->bT32, c->dT32, true);
        pT(c->dT32, c->t132, c->bp32);
        amg_vcycle32(c, c->hp, c->t132, c->dp32, true);
        break;
    case CPTR_STAGE1_BD:
        amg_vcycle32(c, c->hp, c->bp32, c->dp32, true);
        amg_vcycle32(c, c->hT, c->bT32, c->dT32, true);
        break;
    case CPTR_STAGE1_CPR:
        amg_vcycle32(c, c->hp, c->bp32, c->dp32, true);
        *pdp = c->dp32;
        return;
    }
    *pdp = c->dp32;
    *pdT = c->dT32;
}

static void apply_precond32(const Ctx *c, const double *v, double *z) {
    const float *dp, *dT;
    int pf = prof_begin(c, PF_STAGE1);
    apply_stage1_32(c, v, &dp, &dT);
    prof_end(c, pf);
    if (!dp) {   // no first stage: second stage on v itself
        pf = prof_begin(c, PF_ILU);
        if (c->o.stage2 == CPTR_STAGE2_ILU0) ilu_apply(c, v, z, (const double *)nullptr, (const double *)nullptr);
        else cudaMemcpyAsync(z, v, sizeof(double) * (size_t)c->n * c->b, cudaMemcpyDeviceToDevice, c->stream);
        prof_end(c, pf);
        return;
    }
    pf = prof_begin(c, PF_RESID);
    launch_resid_pt32(c, dp, dT, v, c->b132);
    prof_end(c, pf);
    pf = prof_begin(c, PF_ILU);
    if (c->o.stage2 == CPTR_STAGE2_ILU0) ilu_apply32(c, c->b132, z, dp, dT);
    else (k_add_x1<float><<<nblk(c->n, 256), 256, 0, c->stream>>>(c->n, c->b, c->ps, c->ts, dp, dT, c->b132, z), note_launch());
    prof_end(c, pf);
}

// z = M2^{-1}(v - A' x1) + x1, x1 = M1^{-1} v  (Sec. 3, two-stage preconditioners)
void apply_precond(const Ctx *c, const double *v, double *z) {
    if (c->o.precision == CPTR_PREC_MIXED) {
        apply_precond32(c, v, z);
        return;
    }
    const double *dp, *dT;
    int pf = prof_begin(c, PF_STAGE1);
    apply_stage1(c, v, &dp, &dT);
    prof_end(c, pf);
    const double *b1 = v;
    if (dp) {
        pf = prof_begin(c, PF_RESID);
        launch_bsr_resid_pt(c, dp, dT, v, c->b1);
        prof_end(c, pf);
        b1 = c->b1;
    }
    if (c->o.stage2 == CPTR_STAGE2_ILU0) {
        pf = prof_begin(c, PF_ILU);
        ilu_apply(c, b1, z, dp, dT);
        prof_end(c, pf);
    } else {
        (k_add_x1<double><<<nblk(c->n, 256), 256, 0, c->stream>>>(c->n, c->b, c->ps, c->ts, dp, dT, b1, z), note_launch());
    }
}

// ------------------------------------------------------------------------------------------------
// device address of a member of the device-resident Krylov state
static const double *ks_field(const Ctx *c, size_t off) {
    return reinterpret_cast<const double *>(reinterpret_cast<const char *>(c->ks) + off);
}

template <int PASS>
static void cgs(const Ctx *c, const double *V, int nc, double *w, const double *coef, int fin, int j,
                double rtol = 0.0, int jdev = 0) {
    int64_t nb = (int64_t)c->n * c->b;
    (k_cgs<PASS><<<kRedBlocks, kRedThreads, 0, c->stream>>>(nb, V, nc, w, coef, c->partial, c->ks, fin, j,
                                                          c->o.restart, rtol, jdev), note_launch());
}

// One Arnoldi step with the column index taken from the device state (ks->k): the kernel
// sequence that is captured once per set-up into a CUDA graph and replayed every iteration.
static void arnoldi_step_device_indexed(const Ctx *c) {
    const int64_t nb = (int64_t)c->n * c->b;
    const unsigned vgrid = 4 * 152;
    cudaStream_t s = c->stream;
    (k_copy_col<<<vgrid, 256, 0, s>>>(nb, c->V, c->vcur, c->ks, 0), note_launch());
    apply_precond(c, c->vcur, c->zcur);
    (k_copy_col<<<vgrid, 256, 0, s>>>(nb, c->Z, c->zcur, c->ks, 1), note_launch());
    int pf = prof_begin(c, PF_SPMV);
    launch_bsr_spmv(c, c->zcur, c->w);
    prof_end(c, pf);
    pf = prof_begin(c, PF_ARNOLDI);
    cgs<PASS_DOT>(c, c->V, 0, c->w, nullptr, FIN_H, 0, 0.0, 1);
    cgs<PASS_UPD_DOT>(c, c->V, 0, c->w, ks_field(c, offsetof(KState, h)), FIN_H2, 0, 0.0, 1);
    cgs<PASS_UPD_NORM>(c, c->V, 0, c->w, ks_field(c, offsetof(KState, h2)), FIN_GIVENS, 0, 0.0, 1);
    (k_scale<<<vgrid, 256, 0, s>>>(nb, c->w, c->V, c->ks, 0, 1, 1), note_launch());
    prof_end(c, pf);
}

cptr_status build_iteration_graph(Ctx *c) {
    if (c->graph_exec) {
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
    }
    if (!c->cap_stream) CPTR_CUDA_TRY(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    cudaStream_t orig = c->stream;
    c->stream = c->cap_stream;
    begin_capture_count();
    prof_begin_capture(c);
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        arnoldi_step_device_indexed(c);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(c->cap_stream, &g);
        if (e == cudaSuccess) {
            e = cudaGraphInstantiate(&c->graph_exec, g, 0);
            cudaGraphDestroy(g);
        }
    }
    prof_end_capture(c);
    c->graph_launches = end_capture_count();
    c->graph_mask = c->prof.mask;
    c->graph_inject = c->inject_wait;
    c->stream = orig;
    if (e != cudaSuccess) {
        c->graph_exec = nullptr;
        return c->fail(CPTR_ECUDA, std::string("capture of the Arnoldi step: ") + cudaGetErrorString(e));
    }
    return CPTR_OK;
}

// The condition of the restart cycle's WHILE node, evaluated after every Arnoldi step: go on
// while the cycle has columns left, the solve has steps left and neither convergence, breakdown
// nor a bounded wait that gave up has been recorded.
__global__ void k_cycle_cond(const KState *ks, int m, int max_it, cudaGraphConditionalHandle h) {
    const bool more = !ks->done && !ks->wait_err && ks->k < m && ks->its < max_it;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

// A whole restart cycle as one graph launch: a conditional WHILE node (evaluated on the device)
// whose body is the captured Arnoldi step followed by k_cycle_cond, so the host waits once per
// cycle instead of once per step.  Where conditional nodes are not available the per-step graph
// is used (cycle_failed).
static cptr_status build_cycle_graph(Ctx *c) {
    if (c->cycle_exec) {
        cudaGraphExecDestroy(c->cycle_exec);
        c->cycle_exec = nullptr;
    }
    if (!c->cap_stream) CPTR_CUDA_TRY(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    CPTR_CUDA_TRY(c, cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    cudaGraph_t body = nullptr;
    if (e == cudaSuccess) {
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = h;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t node;
        e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p);
        if (e == cudaSuccess) body = p.conditional.phGraph_out[0];
    }
    if (e == cudaSuccess) {
        cudaStream_t orig = c->stream;
        c->stream = c->cap_stream;
        begin_capture_count();
        e = cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            arnoldi_step_device_indexed(c);
            (k_cycle_cond<<<1, 1, 0, c->cap_stream>>>(c->ks, c->o.restart, c->o.max_it, h), note_launch());
            e = cudaStreamEndCapture(c->cap_stream, &body);
        }
        c->cycle_step_launches = end_capture_count();
        c->stream = orig;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->cycle_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->cycle_exec = nullptr;
        c->cycle_failed = true;
    }
    return CPTR_OK;
}

static cptr_status read_state(Ctx *c) {
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->ks_host, c->ks, offsetof(KState, h), cudaMemcpyDeviceToHost, c->stream));
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return CPTR_OK;
}

cptr_status fgmres_solve(Ctx *c, const double *bw, double *x, double rtol, cptr_stats *st) {
    const int m = c->o.restart;
    const int64_t nb = (int64_t)c->n * c->b;
    cudaStream_t s = c->stream;
    const unsigned vgrid = 4 * 152;
    // a whole cycle per launch when nothing is timed per kernel family (event nodes may not sit in
    // a conditional body) and no wait failure is injected; otherwise one graph per step
    const bool cycle = c->o.use_graph == 1 && c->prof.mask == 0 && !c->inject_wait && !c->cycle_failed;
    if (cycle && !c->cycle_exec) CPTR_TRY(build_cycle_graph(c));
    if (c->o.use_graph && !(cycle && c->cycle_exec) &&
        (!c->graph_exec || c->graph_mask != c->prof.mask || c->graph_inject != c->inject_wait))
        CPTR_TRY(build_iteration_graph(c));
    if (!c->o.use_graph && c->graph_exec) {
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
    }
    CPTR_CUDA_TRY(c, cudaMemsetAsync(c->ks, 0, sizeof(KState), s));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(x, 0, sizeof(double) * nb, s));
    // ||b'||, beta = ||b'|| (x = 0), v_0 = b' / beta
    cgs<PASS_NORM>(c, nullptr, 0, const_cast<double *>(bw), nullptr, FIN_BNORM, 0, rtol);
    CPTR_TRY(read_state(c));
    int it = 0, restarts = 0;
    bool done = c->ks_host->done != 0;
    if (!done) (k_scale<<<vgrid, 256, 0, s>>>(nb, bw, c->V, c->ks, 1, 0, 0), note_launch());
    while (!done) {
        int every = c->o.check_every > 0 ? c->o.check_every : 1;
        if (cycle && c->cycle_exec && it < c->o.max_it) {   // the whole cycle, one launch
            CPTR_CUDA_TRY(c, cudaGraphLaunch(c->cycle_exec, s));
            CPTR_TRY(read_state(c));
            note_launches((int64_t)c->ks_host->k * c->cycle_step_launches);
            it = c->ks_host->its;
            if (c->ks_host->wait_err) return c->fail(CPTR_ETIMEOUT, "ILU(0) sweep: a bounded wait gave up");
        }
        for (int j = 0; j < m && it < c->o.max_it && !(cycle && c->cycle_exec); ++j) {
            if (c->graph_exec) {
                CPTR_CUDA_TRY(c, cudaGraphLaunch(c->graph_exec, s));
                note_launches(c->graph_launches);
                ++it;
                CPTR_TRY(read_state(c));
                CPTR_TRY(prof_collect_graph(c));
                if (c->ks_host->wait_err) return c->fail(CPTR_ETIMEOUT, "ILU(0) sweep: a bounded wait gave up");
                if (c->ks_host->done) break;
                continue;
            }
            double *vj = c->V + (int64_t)j * nb, *zj = c->Z + (int64_t)j * nb;
            apply_precond(c, vj, zj);
            int pf = prof_begin(c, PF_SPMV);
            launch_bsr_spmv(c, zj, c->w);
            prof_end(c, pf);
            pf = prof_begin(c, PF_ARNOLDI);
            cgs<PASS_DOT>(c, c->V, j + 1, c->w, nullptr, FIN_H, j);
            cgs<PASS_UPD_DOT>(c, c->V, j + 1, c->w, ks_field(c, offsetof(KState, h)), FIN_H2, j);
            cgs<PASS_UPD_NORM>(c, c->V, j + 1, c->w, ks_field(c, offsetof(KState, h2)), FIN_GIVENS, j);
            (k_scale<<<vgrid, 256, 0, s>>>(nb, c->w, c->V + (int64_t)(j + 1) * nb, c->ks, 0, 1, 0), note_launch());
            prof_end(c, pf);
            ++it;
            if (it % every == 0 || j == m - 1 || it >= c->o.max_it) {
                CPTR_TRY(read_state(c));
                if (c->ks_host->wait_err) return c->fail(CPTR_ETIMEOUT, "ILU(0) sweep: a bounded wait gave up");
                if (c->ks_host->done) break;
            }
        }
        CPTR_CUDA_TRY(c, cudaGetLastError());
        CPTR_TRY(read_state(c));
        if (c->ks_host->breakdown) break;
        (k_trisolve<<<1, 32, 0, s>>>(c->ks, m), note_launch());
        (k_update_x<<<vgrid, 256, 0, s>>>(nb, c->Z, c->ks, x), note_launch());
        if (c->ks_host->done || it >= c->o.max_it) break;
        // restart: r = b' - A' x, beta = ||r||, v_0 = r / beta
        launch_bsr_resid(c, x, bw, c->w);
        cgs<PASS_NORM>(c, nullptr, 0, c->w, nullptr, FIN_RESTART, 0);
        CPTR_TRY(read_state(c));
        if (c->ks_host->done) break;
        (k_scale<<<vgrid, 256, 0, s>>>(nb, c->w, c->V, c->ks, 1, 0, 0), note_launch());
        ++restarts;
    }
    // true residual
    launch_bsr_resid(c, x, bw, c->w);
    cgs<PASS_NORM>(c, nullptr, 0, c->w, nullptr, FIN_TRUE, 0);
    CPTR_CUDA_TRY(c, cudaGetLastError());
    CPTR_TRY(read_state(c));
    const KState &h = *c->ks_host;
    if (h.wait_err) return c->fail(CPTR_ETIMEOUT, "ILU(0) sweep: a bounded wait gave up");
    if (st) {
        st->iters = it;
        st->restarts = restarts;
        st->converged = h.done && !h.breakdown;
        st->est_rel_res = h.est;
        st->bnorm = h.bnorm;
        st->true_rel_res = h.bnorm > 0.0 ? h.true_res / h.bnorm : 0.0;
    }
    if (h.breakdown) return c->fail(CPTR_EBREAKDOWN, "FGMRES: non-finite value in the Arnoldi process");
    return (h.done) ? CPTR_OK : CPTR_NOT_CONVERGED;
}

// ------------------------------------------------------------------------------------------------
// Ensemble: independent instances set up as one block-diagonal system.  The preconditioner and
// the outer SpMV act on the union (they are block diagonal, so each instance's block sees only its
// own values); FGMRES runs per instance.  The union vector is cut into tiles that never straddle
// two instances; one block per tile.  Every instance has its own KState: its own column index,
// Givens rotations, convergence test and step count, and a per-instance last-block reduction
// over its own tiles (in tile order: deterministic).  Instances advance in lockstep; one that has
// converged is skipped by the Gram-Schmidt kernels until the others finish.

// One Gram-Schmidt pass per instance (same passes as k_cgs), column index from the instance state
template <int PASS>
__global__ void __launch_bounds__(kRedThreads) k_bcgs(int64_t nb, const double *__restrict__ V, double *__restrict__ w,
                                                     int coef_off, double *__restrict__ partial, KState *ksb,
                                                     const int32_t *__restrict__ tile_inst,
                                                     const int64_t *__restrict__ tile_beg,
                                                     const int32_t *__restrict__ inst_tile0, int fin, int m,
                                                     double rtol) {
    __shared__ double scoef[kMaxC];
    __shared__ double red[kRedThreads / 32][kMaxC];
    __shared__ bool last;
    const int inst = tile_inst[blockIdx.x];
    KState *ks = ksb + inst;
    // converged instances skip the Arnoldi passes and the restart; FIN_BNORM / FIN_TRUE run for all
    if (ks->done && (fin <= FIN_GIVENS || fin == FIN_RESTART)) return;
    const int j = ks->k, nc = j + 1;
    constexpr bool UPD = PASS == PASS_UPD_DOT || PASS == PASS_UPD_NORM;
    constexpr bool NORM = PASS == PASS_UPD_NORM || PASS == PASS_NORM;
    if (UPD && threadIdx.x < kMaxC) {
        const double *coef = reinterpret_cast<const double *>(reinterpret_cast<const char *>(ks) + coef_off);
        scoef[threadIdx.x] = threadIdx.x < nc ? coef[threadIdx.x] : 0.0;
    }
    __syncthreads();
    const int64_t beg = tile_beg[blockIdx.x], end = tile_beg[blockIdx.x + 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int na = NORM ? 1 : nc;
    cgs_dispatch<PASS>(beg + threadIdx.x, end, blockDim.x, nb, V, nc, w, scoef, red, lane, wid);
    __syncthreads();
    if (threadIdx.x < na) {
        double sum = 0.0;
        for (int w8 = 0; w8 < kRedThreads / 32; ++w8) sum += red[w8][threadIdx.x];
        partial[(int64_t)blockIdx.x * kPStride + threadIdx.x] = sum;
    }
    __threadfence();
    __syncthreads();
    const int t0 = inst_tile0[inst], t1 = inst_tile0[inst + 1];
    if (threadIdx.x == 0) last = atomicAdd(&ks->ticket, 1u) == (unsigned)(t1 - t0 - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double res[kMaxC];
    constexpr int kPU = 8;   // partials per lane in one batch of loads (then added in block order)
    for (int q = wid; q < na; q += kRedThreads / 32) {
        double sum = 0.0;
        for (int b0 = t0 + lane; b0 < t1; b0 += 32 * kPU) {
            double pv[kPU];
#pragma unroll
            for (int u = 0; u < kPU; ++u)
                pv[u] = b0 + 32 * u < t1 ? __ldcg(partial + (int64_t)(b0 + 32 * u) * kPStride + q) : 0.0;
#pragma unroll
            for (int u = 0; u < kPU; ++u)
                if (b0 + 32 * u < t1) sum += pv[u];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
        if (lane == 0) res[q] = sum;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    ks->ticket = 0;
    cgs_finish(ks, res, fin, j, m, rtol, nc);
}

// dst = src / scale per instance (scale = hnorm (which 0) or beta (which 1)); jdev: dst is the
// instance's column k
__global__ void k_bscale(int64_t nb, const double *__restrict__ src, double *__restrict__ dst, const KState *ksb,
                         const int32_t *__restrict__ tile_inst, const int64_t *__restrict__ tile_beg, int which,
                         int jdev) {
    const KState *ks = ksb + tile_inst[blockIdx.x];
    if (ks->done) return;
    if (jdev) dst += (int64_t)ks->k * nb;
    const double sc = which == 0 ? ks->hnorm : ks->beta;
    if (!(sc > 0.0)) return;
    const double inv = 1.0 / sc;
    const int64_t beg = tile_beg[blockIdx.x], end = tile_beg[blockIdx.x + 1];
    for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) dst[i] = src[i] * inv;
}

// vec <-> column k of each instance (dir 0: vec = base[k]; dir 1: base[k] = vec).  Converged
// instances are skipped: their k may equal m (converged on the last step of a cycle), and Z has
// only m columns; their tiles of vec keep the last (finite) values
__global__ void k_bcopy_col(int64_t nb, double *__restrict__ base, double *__restrict__ vec, const KState *ksb,
                            const int32_t *__restrict__ tile_inst, const int64_t *__restrict__ tile_beg, int dir) {
    const KState *ks = ksb + tile_inst[blockIdx.x];
    if (ks->done) return;
    const double *colr = base + (int64_t)ks->k * nb;
    double *colw = base + (int64_t)ks->k * nb;
    const int64_t beg = tile_beg[blockIdx.x], end = tile_beg[blockIdx.x + 1];
    for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
        if (dir == 0) vec[i] = colr[i];
        else colw[i] = vec[i];
    }
}

// y = H^{-1} g for every instance that iterated in this cycle (one thread per instance)
__global__ void k_btrisolve(KState *ksb, int n_inst, int m) {
    const int inst = blockIdx.x * blockDim.x + threadIdx.x;
    if (inst >= n_inst) return;
    KState *ks = ksb + inst;
    if (!ks->active) return;
    const int k = ks->k;
    for (int i = k - 1; i >= 0; --i) {
        double sum = ks->g[i];
        for (int q = i + 1; q < k; ++q) sum -= ks->H[(int64_t)q * (m + 1) + i] * ks->y[q];
        ks->y[i] = sum / ks->H[(int64_t)i * (m + 1) + i];
    }
}

// x += sum_{q < k} y_q z_q on the tiles of the instances that iterated in this cycle
__global__ void __launch_bounds__(256) k_bupdate_x(int64_t nb, const double *__restrict__ Z, const KState *ksb,
                                                   const int32_t *__restrict__ tile_inst,
                                                   const int64_t *__restrict__ tile_beg, double *__restrict__ x) {
    __shared__ double sy[kMaxC];
    const KState *ks = ksb + tile_inst[blockIdx.x];
    if (!ks->active) return;
    const int k = ks->k;
    if (threadIdx.x < kMaxC) sy[threadIdx.x] = threadIdx.x < k ? ks->y[threadIdx.x] : 0.0;
    __syncthreads();
    const int64_t beg = tile_beg[blockIdx.x], end = tile_beg[blockIdx.x + 1];
    for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
        double sum = x[i];
#pragma unroll
        for (int q = 0; q < kMaxC; ++q)
            if (q < k) sum = fma(sy[q], __ldg(Z + (int64_t)q * nb + i), sum);
        x[i] = sum;
    }
}

// end of a cycle: no instance is active until its restart
__global__ void k_bend_cycle(KState *ksb, int n_inst) {
    const int inst = blockIdx.x * blockDim.x + threadIdx.x;
    if (inst < n_inst) ksb[inst].active = 0;
}

// compact copy of the instance headers (and, last, the ILU wait flag of the shared state)
__global__ void k_bheaders(const KState *ksb, int n_inst, const KState *ks, KHdr *hdr) {
    const int inst = blockIdx.x * blockDim.x + threadIdx.x;
    if (inst < n_inst) memcpy(hdr + inst, ksb + inst, sizeof(KHdr));
    if (inst == 0) {
        memset(hdr + n_inst, 0, sizeof(KHdr));
        hdr[n_inst].wait_err = ks->wait_err;
    }
}

namespace {

template <int PASS>
void bcgs(const Ctx *c, const double *V, double *w, size_t coef_off, int fin, double rtol = 0.0) {
    const int64_t nb = (int64_t)c->n * c->b;
    (k_bcgs<PASS><<<c->n_tiles, kRedThreads, 0, c->stream>>>(nb, V, w, (int)coef_off, c->partial_b, c->ksb,
                                                             c->tile_inst, c->tile_beg, c->inst_tile0, fin,
                                                             c->o.restart, rtol), note_launch());
}

void bheaders(const Ctx *c) {
    (k_bheaders<<<nblk(c->n_inst, 64), 64, 0, c->stream>>>(c->ksb, c->n_inst, c->ks, c->hdr), note_launch());
}

// one Arnoldi step of every instance (captured once per set-up, replayed every iteration)
void arnoldi_step_batch(const Ctx *c) {
    const int64_t nb = (int64_t)c->n * c->b;
    cudaStream_t s = c->stream;
    const unsigned T = c->n_tiles;
    (k_bcopy_col<<<T, 256, 0, s>>>(nb, c->V, c->vcur, c->ksb, c->tile_inst, c->tile_beg, 0), note_launch());
    apply_precond(c, c->vcur, c->zcur);
    (k_bcopy_col<<<T, 256, 0, s>>>(nb, c->Z, c->zcur, c->ksb, c->tile_inst, c->tile_beg, 1), note_launch());
    launch_bsr_spmv(c, c->zcur, c->w);
    bcgs<PASS_DOT>(c, c->V, c->w, 0, FIN_H);
    bcgs<PASS_UPD_DOT>(c, c->V, c->w, offsetof(KState, h), FIN_H2);
    bcgs<PASS_UPD_NORM>(c, c->V, c->w, offsetof(KState, h2), FIN_GIVENS);
    (k_bscale<<<T, 256, 0, s>>>(nb, c->w, c->V, c->ksb, c->tile_inst, c->tile_beg, 0, 1), note_launch());
    bheaders(c);
}

cptr_status build_batch_graph(Ctx *c) {
    if (c->bgraph_exec) {
        cudaGraphExecDestroy(c->bgraph_exec);
        c->bgraph_exec = nullptr;
    }
    if (!c->cap_stream) CPTR_CUDA_TRY(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    cudaStream_t orig = c->stream;
    c->stream = c->cap_stream;
    const uint32_t mask = c->prof.mask;
    c->prof.mask = 0;   // no event timing inside the ensemble graph
    begin_capture_count();
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        arnoldi_step_batch(c);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(c->cap_stream, &g);
        if (e == cudaSuccess) {
            e = cudaGraphInstantiate(&c->bgraph_exec, g, 0);
            cudaGraphDestroy(g);
        }
    }
    c->bgraph_launches = end_capture_count();
    c->prof.mask = mask;
    c->stream = orig;
    if (e != cudaSuccess) {
        c->bgraph_exec = nullptr;
        return c->fail(CPTR_ECUDA, std::string("capture of the ensemble Arnoldi step: ") + cudaGetErrorString(e));
    }
    return CPTR_OK;
}

// The condition of the ensemble cycle's WHILE node, after every lockstep step: count the step
// (ks->k steps in this cycle, ks->its in the solve, mirrored into the shared header) and go on
// while an instance still iterates in this cycle, the cycle and the solve have steps left and no
// bounded wait gave up.
__global__ void k_bcycle_cond(const KState *ksb, int n_inst, KState *ks, KHdr *hdr, int m, int max_it,
                              cudaGraphConditionalHandle h) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    bool a = false;
    for (int i = threadIdx.x; i < n_inst; i += blockDim.x) a |= ksb[i].active && !ksb[i].done;
    if (a) atomicOr(&any, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        ks->k += 1;
        ks->its += 1;
        hdr[n_inst].k = ks->k;
        hdr[n_inst].its = ks->its;
        const bool more = any && !ks->wait_err && ks->k < m && ks->its < max_it;
        cudaGraphSetConditional(h, more ? 1u : 0u);
    }
}

// The ensemble's restart cycle as one graph launch (a conditional WHILE node over the lockstep
// Arnoldi step of every instance); the per-step graph where conditional nodes are not available.
cptr_status build_batch_cycle_graph(Ctx *c) {
    if (c->bcycle_exec) {
        cudaGraphExecDestroy(c->bcycle_exec);
        c->bcycle_exec = nullptr;
    }
    if (!c->cap_stream) CPTR_CUDA_TRY(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    CPTR_CUDA_TRY(c, cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    cudaGraph_t body = nullptr;
    if (e == cudaSuccess) {
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = h;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t node;
        e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p);
        if (e == cudaSuccess) body = p.conditional.phGraph_out[0];
    }
    if (e == cudaSuccess) {
        cudaStream_t orig = c->stream;
        c->stream = c->cap_stream;
        const uint32_t mask = c->prof.mask;
        c->prof.mask = 0;
        begin_capture_count();
        e = cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            arnoldi_step_batch(c);
            (k_bcycle_cond<<<1, 256, 0, c->cap_stream>>>(c->ksb, c->n_inst, c->ks, c->hdr, c->o.restart, c->o.max_it, h),
             note_launch());
            e = cudaStreamEndCapture(c->cap_stream, &body);
        }
        c->bcycle_step_launches = end_capture_count();
        c->prof.mask = mask;
        c->stream = orig;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->bcycle_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->bcycle_exec = nullptr;
        c->bcycle_failed = true;
    }
    return CPTR_OK;
}

cptr_status read_headers(Ctx *c) {
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->hdr_host, c->hdr, sizeof(KHdr) * (c->n_inst + 1), cudaMemcpyDeviceToHost,
                                     c->stream));
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return CPTR_OK;
}

}  // namespace

void free_batch(Ctx *c) {
    dfree(c->tile_inst); dfree(c->tile_beg); dfree(c->inst_tile0); dfree(c->ksb); dfree(c->hdr);
    dfree(c->partial_b);
    c->tile_inst = nullptr; c->tile_beg = nullptr; c->inst_tile0 = nullptr; c->ksb = nullptr; c->hdr = nullptr;
    c->partial_b = nullptr;
    if (c->hdr_host) cudaFreeHost(c->hdr_host);
    c->hdr_host = nullptr;
    if (c->bgraph_exec) cudaGraphExecDestroy(c->bgraph_exec);
    c->bgraph_exec = nullptr;
    if (c->bcycle_exec) cudaGraphExecDestroy(c->bcycle_exec);
    c->bcycle_exec = nullptr;
    c->n_inst = 0;
    c->n_tiles = 0;
    c->inst_cell0.clear();
}

cptr_status fgmres_solve_batch(Ctx *c, const double *bw, double *x, double rtol, cptr_stats *st) {
    const int m = c->o.restart, ni = c->n_inst;
    const int64_t nb = (int64_t)c->n * c->b;
    cudaStream_t s = c->stream;
    const unsigned T = c->n_tiles;
    const bool cycle = c->o.use_graph == 1 && !c->inject_wait && !c->bcycle_failed;
    if (cycle && !c->bcycle_exec) CPTR_TRY(build_batch_cycle_graph(c));
    if (!(cycle && c->bcycle_exec) && !c->bgraph_exec) CPTR_TRY(build_batch_graph(c));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(c->ksb, 0, sizeof(KState) * ni, s));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(c->ks, 0, sizeof(KState), s));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(x, 0, sizeof(double) * nb, s));
    bcgs<PASS_NORM>(c, nullptr, const_cast<double *>(bw), 0, FIN_BNORM, rtol);
    (k_bscale<<<T, 256, 0, s>>>(nb, bw, c->V, c->ksb, c->tile_inst, c->tile_beg, 1, 0), note_launch());
    bheaders(c);
    CPTR_TRY(read_headers(c));
    std::vector<int32_t> restarts(ni, 0);
    auto all_done = [&]() {
        for (int i = 0; i < ni; ++i)
            if (!c->hdr_host[i].done) return false;
        return true;
    };
    auto none_active = [&]() {
        for (int i = 0; i < ni; ++i)
            if (c->hdr_host[i].active && !c->hdr_host[i].done) return false;
        return true;
    };
    int it = 0;
    bool stop = all_done();
    while (!stop) {
        if (cycle && c->bcycle_exec && it < c->o.max_it) {   // the whole cycle, one launch
            CPTR_CUDA_TRY(c, cudaMemsetAsync(&c->ks->k, 0, sizeof(int32_t), s));
            CPTR_CUDA_TRY(c, cudaGraphLaunch(c->bcycle_exec, s));
            CPTR_TRY(read_headers(c));
            note_launches((int64_t)c->hdr_host[ni].k * c->bcycle_step_launches);
            it = c->hdr_host[ni].its;
            if (c->hdr_host[ni].wait_err) return c->fail(CPTR_ETIMEOUT, "ILU(0) sweep: a bounded wait gave up");
        }
        for (int j = 0; j < m && it < c->o.max_it && !(cycle && c->bcycle_exec); ++j) {
            CPTR_CUDA_TRY(c, cudaGraphLaunch(c->bgraph_exec, s));
            note_launches(c->bgraph_launches);
            ++it;
            CPTR_TRY(read_headers(c));
            if (c->hdr_host[ni].wait_err) return c->fail(CPTR_ETIMEOUT, "ILU(0) sweep: a bounded wait gave up");
            if (none_active()) break;
        }
        (k_btrisolve<<<nblk(ni, 64), 64, 0, s>>>(c->ksb, ni, m), note_launch());
        (k_bupdate_x<<<T, 256, 0, s>>>(nb, c->Z, c->ksb, c->tile_inst, c->tile_beg, x), note_launch());
        (k_bend_cycle<<<nblk(ni, 64), 64, 0, s>>>(c->ksb, ni), note_launch());
        bheaders(c);
        CPTR_TRY(read_headers(c));
        if (all_done() || it >= c->o.max_it) break;
        // restart the instances that have not converged: r = b' - A' x, beta, v_0 = r / beta
        for (int i = 0; i < ni; ++i)
            if (!c->hdr_host[i].done) ++restarts[i];
        launch_bsr_resid(c, x, bw, c->w);
        bcgs<PASS_NORM>(c, nullptr, c->w, 0, FIN_RESTART);
        (k_bscale<<<T, 256, 0, s>>>(nb, c->w, c->V, c->ksb, c->tile_inst, c->tile_beg, 1, 0), note_launch());
        bheaders(c);
        CPTR_TRY(read_headers(c));
        stop = all_done();
    }
    // true residual of every instance
    launch_bsr_resid(c, x, bw, c->w);
    bcgs<PASS_NORM>(c, nullptr, c->w, 0, FIN_TRUE);
    bheaders(c);
    CPTR_CUDA_TRY(c, cudaGetLastError());
    CPTR_TRY(read_headers(c));
    if (c->hdr_host[ni].wait_err) return c->fail(CPTR_ETIMEOUT, "ILU(0) sweep: a bounded wait gave up");
    bool conv = true, brk = false;
    for (int i = 0; i < ni; ++i) {
        const KHdr &h = c->hdr_host[i];
        if (st) {
            st[i].iters = h.its;
            st[i].restarts = restarts[i];
            st[i].converged = h.done && !h.breakdown;
            st[i].est_rel_res = h.est;
            st[i].bnorm = h.bnorm;
            st[i].true_rel_res = h.bnorm > 0.0 ? h.true_res / h.bnorm : 0.0;
        }
        conv = conv && h.done && !h.breakdown;
        brk = brk || h.breakdown;
    }
    if (brk) return c->fail(CPTR_EBREAKDOWN, "FGMRES: non-finite value in the Arnoldi process of an instance");
    return conv ? CPTR_OK : CPTR_NOT_CONVERGED;
}

}  // namespace cptr
