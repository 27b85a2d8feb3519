// Second stage of CPR/CPTR: block ILU(0) of the decoupled Jacobian A' on its own BSR pattern
// (Sec. 3.1, Sec. 4: "ILU(0) is our default").  Factorisation and triangular solves are level
// scheduled: level(i) = 1 + max level(j) over the rows j that row i depends on, so rows of one
// level are independent.  Pivot blocks are stored inverted in the diagonal slots.  With dense
// b x b blocks this is the same operator as scalar ILU(0) of the interleaved matrix.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace cptr {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// in-place inverse of a B x B block (Gauss-Jordan, partial pivoting); false if singular
template <int B>
__device__ __forceinline__ bool block_inverse(double *m) {
    double a[B][2 * B];
#pragma unroll
    for (int r = 0; r < B; ++r)
#pragma unroll
        for (int q = 0; q < 2 * B; ++q) a[r][q] = q < B ? m[r * B + q] : (q - B == r ? 1.0 : 0.0);
#pragma unroll
    for (int k = 0; k < B; ++k) {
        int p = k;
        double best = fabs(a[k][k]);
#pragma unroll
        for (int r = k + 1; r < B; ++r)
            if (fabs(a[r][k]) > best) { best = fabs(a[r][k]); p = r; }
        if (best == 0.0) return false;
        if (p != k)
#pragma unroll
            for (int q = 0; q < 2 * B; ++q) { double t = a[k][q]; a[k][q] = a[p][q]; a[p][q] = t; }
        double d = 1.0 / a[k][k];
#pragma unroll
        for (int q = 0; q < 2 * B; ++q) a[k][q] *= d;
#pragma unroll
        for (int r = 0; r < B; ++r) {
            if (r == k) continue;
            double f = a[r][k];
#pragma unroll
            for (int q = 0; q < 2 * B; ++q) a[r][q] = fma(-f, a[k][q], a[r][q]);
        }
    }
#pragma unroll
    for (int r = 0; r < B; ++r)
#pragma unroll
        for (int q = 0; q < B; ++q) m[r * B + q] = a[r][B + q];
    return true;
}

template <int B>
__global__ void k_bilu_factor(const int32_t *rows, int32_t start, int32_t count, const int32_t *rp,
                              const int32_t *ci, const int32_t *diag, double *LU, int32_t *singular) {
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    int32_t i = rows[start + t];
    int32_t e = rp[i + 1];
    for (int32_t k = rp[i]; k < diag[i]; ++k) {
        int32_t c = ci[k];
        const double *dinv = LU + (int64_t)diag[c] * B * B;
        double a[B * B], l[B * B];
#pragma unroll
        for (int q = 0; q < B * B; ++q) a[q] = LU[(int64_t)k * B * B + q];
#pragma unroll
        for (int r = 0; r < B; ++r)
#pragma unroll
            for (int q = 0; q < B; ++q) {
                double s = 0.0;
#pragma unroll
                for (int u = 0; u < B; ++u) s = fma(a[r * B + u], dinv[u * B + q], s);
                l[r * B + q] = s;
            }
#pragma unroll
        for (int q = 0; q < B * B; ++q) LU[(int64_t)k * B * B + q] = l[q];
        int32_t p = k + 1;
        for (int32_t qq = diag[c] + 1; qq < rp[c + 1]; ++qq) {
            int32_t j = ci[qq];
            while (p < e && ci[p] < j) ++p;
            if (p < e && ci[p] == j) {
                const double *u = LU + (int64_t)qq * B * B;
                double *dst = LU + (int64_t)p * B * B;
#pragma unroll
                for (int r = 0; r < B; ++r)
#pragma unroll
                    for (int q = 0; q < B; ++q) {
                        double s = dst[r * B + q];
#pragma unroll
                        for (int w = 0; w < B; ++w) s = fma(-l[r * B + w], u[w * B + q], s);
                        dst[r * B + q] = s;
                    }
            }
        }
    }
    double d[B * B];
    double *dd = LU + (int64_t)diag[i] * B * B;
#pragma unroll
    for (int q = 0; q < B * B; ++q) d[q] = dd[q];
    if (!block_inverse<B>(d)) { atomicOr(singular, 1); return; }
#pragma unroll
    for (int q = 0; q < B * B; ++q) dd[q] = d[q];
}

// forward: y_i = r_i - sum_{k < i} L_ik y_k
template <int B>
__global__ void k_ilu_fwd(const int32_t *__restrict__ rows, int32_t start, int32_t count,
                          const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                          const int32_t *__restrict__ diag, const double *__restrict__ LU,
                          const double *__restrict__ r, double *__restrict__ y) {
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    int32_t i = rows[start + t];
    double s[B];
#pragma unroll
    for (int q = 0; q < B; ++q) s[q] = r[(int64_t)i * B + q];
    for (int32_t k = rp[i]; k < diag[i]; ++k) {
        int32_t c = ci[k];
        const double *l = LU + (int64_t)k * B * B;
        double yc[B];
#pragma unroll
        for (int q = 0; q < B; ++q) yc[q] = y[(int64_t)c * B + q];
#pragma unroll
        for (int rr = 0; rr < B; ++rr)
#pragma unroll
            for (int q = 0; q < B; ++q) s[rr] = fma(-l[rr * B + q], yc[q], s[rr]);
    }
#pragma unroll
    for (int q = 0; q < B; ++q) y[(int64_t)i * B + q] = s[q];
}

// backward: z_i = D_i^{-1} (y_i - sum_{k > i} U_ik z_k); out_i = z_i + x1_i (x1 from dp, dT)
template <int B>
__global__ void k_ilu_bwd(const int32_t *__restrict__ rows, int32_t start, int32_t count,
                          const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                          const int32_t *__restrict__ diag, const double *__restrict__ LU,
                          const double *__restrict__ y, double *__restrict__ z, double *__restrict__ out, int ps,
                          int ts, const double *__restrict__ dp, const double *__restrict__ dT) {
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    int32_t i = rows[start + t];
    double s[B];
#pragma unroll
    for (int q = 0; q < B; ++q) s[q] = y[(int64_t)i * B + q];
    for (int32_t k = diag[i] + 1; k < rp[i + 1]; ++k) {
        int32_t c = ci[k];
        const double *u = LU + (int64_t)k * B * B;
        double zc[B];
#pragma unroll
        for (int q = 0; q < B; ++q) zc[q] = z[(int64_t)c * B + q];
#pragma unroll
        for (int rr = 0; rr < B; ++rr)
#pragma unroll
            for (int q = 0; q < B; ++q) s[rr] = fma(-u[rr * B + q], zc[q], s[rr]);
    }
    const double *dinv = LU + (int64_t)diag[i] * B * B;
    double zi[B];
#pragma unroll
    for (int rr = 0; rr < B; ++rr) {
        double a = 0.0;
#pragma unroll
        for (int q = 0; q < B; ++q) a = fma(dinv[rr * B + q], s[q], a);
        zi[rr] = a;
    }
#pragma unroll
    for (int q = 0; q < B; ++q) z[(int64_t)i * B + q] = zi[q];
    if (out) {
#pragma unroll
        for (int q = 0; q < B; ++q) {
            double add = 0.0;
            if (dp && q == ps) add = dp[i];
            if (dT && q == ts) add = dT[i];
            out[(int64_t)i * B + q] = zi[q] + add;
        }
    }
}

static void level_sets(int32_t n, const std::vector<int32_t> &rp, const std::vector<int32_t> &ci, bool forward,
                       std::vector<int32_t> &lptr, std::vector<int32_t> &rows) {
    std::vector<int32_t> lev(n, 0);
    int32_t nl = 0;
    for (int32_t s = 0; s < n; ++s) {
        int32_t i = forward ? s : n - 1 - s;
        int32_t l = 0;
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
            int32_t j = ci[k];
            if (forward ? (j < i) : (j > i)) l = std::max(l, lev[j] + 1);
        }
        lev[i] = l;
        nl = std::max(nl, l + 1);
    }
    lptr.assign(nl + 1, 0);
    for (int32_t i = 0; i < n; ++i) lptr[lev[i] + 1]++;
    for (int32_t l = 0; l < nl; ++l) lptr[l + 1] += lptr[l];
    std::vector<int32_t> cur(lptr.begin(), lptr.end() - 1);
    rows.assign(n, 0);
    for (int32_t i = 0; i < n; ++i) rows[cur[lev[i]]++] = i;  // ascending within a level
}

cptr_status ilu_setup(Ctx *c) {
    ilu_free(c);
    std::vector<int32_t> rows_f, rows_b;
    level_sets(c->n, c->h_rp, c->h_ci, true, c->h_lptr_f, rows_f);
    level_sets(c->n, c->h_rp, c->h_ci, false, c->h_lptr_b, rows_b);
    c->nlev_f = (int32_t)c->h_lptr_f.size() - 1;
    c->nlev_b = (int32_t)c->h_lptr_b.size() - 1;
    CPTR_TRY(dalloc_t(c, &c->lvl_f, (size_t)c->n));
    CPTR_TRY(dalloc_t(c, &c->lvl_b, (size_t)c->n));
    CPTR_TRY(dalloc_t(c, &c->LU, (size_t)c->nnzb * c->b * c->b));
    CPTR_TRY(dalloc_t(c, &c->ybuf, (size_t)c->n * c->b));
    CPTR_TRY(dalloc_t(c, &c->zbuf, (size_t)c->n * c->b));
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->lvl_f, rows_f.data(), sizeof(int32_t) * c->n, cudaMemcpyHostToDevice, c->stream));
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->lvl_b, rows_b.data(), sizeof(int32_t) * c->n, cudaMemcpyHostToDevice, c->stream));
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->LU, c->A, sizeof(double) * (size_t)c->nnzb * c->b * c->b,
                                     cudaMemcpyDeviceToDevice, c->stream));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(c->flag, 0, sizeof(int32_t), c->stream));
    for (int32_t l = 0; l < c->nlev_f; ++l) {
        int32_t s = c->h_lptr_f[l], cnt = c->h_lptr_f[l + 1] - s;
        if (c->b == 3)
            (k_bilu_factor<3><<<nblk(cnt, 128), 128, 0, c->stream>>>(c->lvl_f, s, cnt, c->rp, c->ci, c->diag, c->LU, c->flag), note_launch());
        else
            (k_bilu_factor<4><<<nblk(cnt, 128), 128, 0, c->stream>>>(c->lvl_f, s, cnt, c->rp, c->ci, c->diag, c->LU, c->flag), note_launch());
    }
    CPTR_CUDA_TRY(c, cudaGetLastError());
    int32_t sing = 0;
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(&sing, c->flag, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (sing) return c->fail(CPTR_ESINGULAR, "ILU(0): singular pivot block");
    return CPTR_OK;
}

void ilu_free(Ctx *c) {
    dfree(c->lvl_f); dfree(c->lvl_b); dfree(c->LU); dfree(c->ybuf); dfree(c->zbuf);
    c->lvl_f = c->lvl_b = nullptr;
    c->LU = c->ybuf = c->zbuf = nullptr;
}

// z = (LU)^{-1} r + x1, where x1 carries dp in slot ps and dT in slot ts (either may be null)
void ilu_apply(const Ctx *c, const double *r, double *z, const double *dp, const double *dT) {
    cudaStream_t s = c->stream;
    for (int32_t l = 0; l < c->nlev_f; ++l) {
        int32_t st = c->h_lptr_f[l], cnt = c->h_lptr_f[l + 1] - st;
        if (c->b == 3) (k_ilu_fwd<3><<<nblk(cnt, 128), 128, 0, s>>>(c->lvl_f, st, cnt, c->rp, c->ci, c->diag, c->LU, r, c->ybuf), note_launch());
        else (k_ilu_fwd<4><<<nblk(cnt, 128), 128, 0, s>>>(c->lvl_f, st, cnt, c->rp, c->ci, c->diag, c->LU, r, c->ybuf), note_launch());
    }
    for (int32_t l = 0; l < c->nlev_b; ++l) {
        int32_t st = c->h_lptr_b[l], cnt = c->h_lptr_b[l + 1] - st;
        if (c->b == 3)
            (k_ilu_bwd<3><<<nblk(cnt, 128), 128, 0, s>>>(c->lvl_b, st, cnt, c->rp, c->ci, c->diag, c->LU, c->ybuf,
                                                         c->zbuf, z, c->ps, c->ts, dp, dT), note_launch());
        else
            (k_ilu_bwd<4><<<nblk(cnt, 128), 128, 0, s>>>(c->lvl_b, st, cnt, c->rp, c->ci, c->diag, c->LU, c->ybuf,
                                                         c->zbuf, z, c->ps, c->ts, dp, dT), note_launch());
    }
}

// z = (LU)^{-1} r with caller-supplied intermediate vectors ybuf, zbuf (n*b doubles each);
// used by the allocation-free entry point
void ilu_apply_into(const Ctx *c, const double *r, double *z, double *ybuf, double *zbuf) {
    cudaStream_t s = c->stream;
    for (int32_t l = 0; l < c->nlev_f; ++l) {
        int32_t st = c->h_lptr_f[l], cnt = c->h_lptr_f[l + 1] - st;
        if (c->b == 3) (k_ilu_fwd<3><<<nblk(cnt, 128), 128, 0, s>>>(c->lvl_f, st, cnt, c->rp, c->ci, c->diag, c->LU, r, ybuf), note_launch());
        else (k_ilu_fwd<4><<<nblk(cnt, 128), 128, 0, s>>>(c->lvl_f, st, cnt, c->rp, c->ci, c->diag, c->LU, r, ybuf), note_launch());
    }
    for (int32_t l = 0; l < c->nlev_b; ++l) {
        int32_t st = c->h_lptr_b[l], cnt = c->h_lptr_b[l + 1] - st;
        if (c->b == 3)
            (k_ilu_bwd<3><<<nblk(cnt, 128), 128, 0, s>>>(c->lvl_b, st, cnt, c->rp, c->ci, c->diag, c->LU, ybuf, zbuf, z,
                                                         c->ps, c->ts, nullptr, nullptr), note_launch());
        else
            (k_ilu_bwd<4><<<nblk(cnt, 128), 128, 0, s>>>(c->lvl_b, st, cnt, c->rp, c->ci, c->diag, c->LU, ybuf, zbuf, z,
                                                         c->ps, c->ts, nullptr, nullptr), note_launch());
    }
}

}  // namespace cptr
