/*
 * FP64 CPU oracle for the CPTR-preconditioned FGMRES solve (arXiv 1907.04229).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, serial, obviously-correct restatement of the
 * method against which the CUDA library is checked.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product path never calls it.  It shares no
 * code with the CUDA library.  Compile with -ffp-contract=off so that results do not depend on
 * whether the target fuses multiply-adds.
 *
 * Data: scalar CSR (int32 indices, double values).  The BSR Jacobian handed to or_create is
 * expanded to the interleaved (cell-major) scalar CSR: unknown u of cell i is row i*b + u.
 *
 * Steps, each with the passage it follows:
 *   decoupling + scaling  A' = W A, b' = W b            Sec. 2.2.2 eq. (weighted), Sec. 3.5 eq. (scaling)
 *   p-T restriction       A_00 = [A_pp A_pT; A_Tp A_TT]  Sec. 3.2 eq. (A00)
 *   block preconditioner  5 steps for A_00^{-1}          Sec. 3.3 eq. (Aschur) and its step list
 *   Schur approximation   S~_T given (eq. Se) or A_TT    Sec. 3.3.1
 *   CPR first stage       A_pp^{-1} on b_p               Sec. 3.1
 *   uAMG first stage      unknown-based AMG V-cycle on A_00 (coarsening and interpolation of each
 *                         diagonal block on its own, Galerkin product and smoothing on the coupled
 *                         A_00)                           Sec. 3.4
 *   S~_diag               A_TT - A_Tp diag(A_pp)^{-1} A_pT   Sec. 3.3.1
 *   QI / TI decoupling    stage 1 solves with S = A_00 - D A_s0 (CPR: A_pp - D A_sp) on the
 *                         decoupled right-hand side R G v, G = [I -D; 0 I], D_QI = diag(A_0s)
 *                         diag(A_ss)^{-1}, D_TI = colsum(A_0s) colsum(A_ss)^{-1}   Sec. 3.1, 3.2
 *   two-stage combination x1 = M1^-1 v, b1 = v - A x1,
 *                         z = M2^-1 b1 + x1              Sec. 3 "Two-stage preconditioners"
 *   second stage          ILU(0), or ILU(1)              Sec. 4 (ILU(0) default; ILU(1) in the
 *                                                        CPR-AMG-ILU(1) comparisons)
 *   AMG V-cycle           strength, PMIS, direct interpolation, Galerkin RAP, l1-Jacobi or
 *                         omega-Jacobi, one pre- and one post-sweep, dense LU on the coarsest
 *                         level (replaces BoomerAMG's defaults, Sec. 4)
 *   Krylov                right-preconditioned (flexible) GMRES, restart m, classical
 *                         Gram-Schmidt with one full re-orthogonalisation, Givens rotations,
 *                         stop when the residual estimate <= rtol * ||b'||      Sec. 3, Sec. 4
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------------ */
/* options and stats (layout mirrored by oracle/__init__.py)                                   */
enum { OR_CPTR_FULL = 0, OR_CPTR_UPPER = 1, OR_CPTR_LOWER = 2, OR_BD = 3, OR_CPR = 4, OR_NONE1 = 5, OR_UAMG = 6 };
enum { OR_ILU0 = 0, OR_NONE2 = 1 };
enum { OR_SCHUR_GIVEN = 0, OR_SCHUR_ATT = 1, OR_SCHUR_DIAG = 3 };
enum { OR_L1 = 0, OR_JACOBI = 1 };

typedef struct {
    int32_t stage1, stage2, schur, smoother;
    double omega, theta;
    int32_t n_coarse, max_levels, restart, max_it;
    int32_t dense_max, seed;
    int32_t ilu_order;       /* 0: natural cell order; 1: multicolour (greedy colouring) */
    int32_t precision;       /* 0: FP64 everywhere; 1: stored preconditioner values rounded as the
                                mixed-precision GPU form stores them (FP64 arithmetic) */
    int32_t decouple;        /* 0: none; 1: Quasi-IMPES; 2: True-IMPES (CPR and uAMG first stages) */
    int32_t ilu_fill;        /* level of fill of the second stage: 0 (ILU(0)) or 1 (ILU(1)) */
    const int32_t *part;     /* part id per cell: block-Jacobi ILU(0) over the parts (Sec. 4), or NULL */
} or_opts;

typedef struct {
    int32_t iters, restarts, converged, pad;
    double est_rel_res, true_rel_res, bnorm;
} or_stats;

typedef struct {
    int32_t n, nnz;
    int32_t *rp, *ci;
    double *v;
} csr;

static void csr_alloc(csr *a, int32_t n, int32_t nnz) {
    a->n = n; a->nnz = nnz;
    a->rp = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    a->ci = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    a->v = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
}
static void csr_free(csr *a) { free(a->rp); free(a->ci); free(a->v); memset(a, 0, sizeof(*a)); }

/* y = A x */
static void spmv(const csr *A, const double *x, double *y) {
    for (int32_t i = 0; i < A->n; ++i) {
        double s = 0.0;
        for (int32_t k = A->rp[i]; k < A->rp[i + 1]; ++k) s += A->v[k] * x[A->ci[k]];
        y[i] = s;
    }
}
static double dot(int64_t n, const double *x, const double *y) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];
    return s;
}

/* ------------------------------------------------------------------------------------------ */
/* AMG                                                                                          */
typedef struct {
    csr A;          /* level operator */
    double *dinv;   /* smoother diagonal inverse */
    csr P, PT;      /* interpolation n x nc and its transpose (empty on the coarsest level) */
    int32_t *cf;    /* 1 = C, 2 = F (empty on the coarsest level) */
    double *r, *x, *b; /* work */
} amg_level;

typedef struct {
    int nlev;
    amg_level L[32];
    double *lu;     /* coarsest: dense LU with partial pivoting (row-major) or NULL */
    int32_t *piv;
    int dense;      /* 1: coarsest level solved by dense LU; 0: by two smoothing sweeps */
} amg;

static uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
    /* i-th (0-based) output of the SplitMix64 stream started at state seed */
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Classical strength: j != i is strong for i iff -a_ij >= theta * max_{k != i}(-a_ik) and the
 * maximum is positive.  Returned as a CSR pattern S (row i lists the j that i depends on). */
static void strength(const csr *A, double theta, int32_t **Srp, int32_t **Sci) {
    int32_t n = A->n;
    int32_t *rp = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    int32_t *ci = (int32_t *)malloc(sizeof(int32_t) * (size_t)(A->nnz > 0 ? A->nnz : 1));
    int32_t cnt = 0;
    for (int32_t i = 0; i < n; ++i) {
        double m = 0.0;
        int have = 0;
        for (int32_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
            if (A->ci[k] == i) continue;
            double t = -A->v[k];
            if (!have || t > m) { m = t; have = 1; }
        }
        if (have && m > 0.0) {
            double thr = theta * m;
            for (int32_t k = A->rp[i]; k < A->rp[i + 1]; ++k)
                if (A->ci[k] != i && -A->v[k] >= thr) ci[cnt++] = A->ci[k];
        }
        rp[i + 1] = cnt;
    }
    *Srp = rp; *Sci = ci;
}

static void transpose_pattern(int32_t n, const int32_t *rp, const int32_t *ci, int32_t **Trp, int32_t **Tci) {
    int32_t nnz = rp[n];
    int32_t *trp = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    int32_t *tci = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    for (int32_t k = 0; k < nnz; ++k) trp[ci[k] + 1]++;
    for (int32_t i = 0; i < n; ++i) trp[i + 1] += trp[i];
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    memcpy(pos, trp, sizeof(int32_t) * ((size_t)n + 1));
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) tci[pos[ci[k]]++] = i; /* rows ascending */
    free(pos);
    *Trp = trp; *Tci = tci;
}

/* key order used by PMIS: (|S^T_i|, 32-bit hash) with the larger index winning exact ties */
static int beats(uint64_t ki, int32_t i, uint64_t kj, int32_t j) { return ki > kj || (ki == kj && i > j); }

/* PMIS C/F splitting (De Sterck, Yang, Heys 2006), round-synchronous.  cf: 1 = C, 2 = F. */
static void pmis(int32_t n, const int32_t *Srp, const int32_t *Sci, uint64_t seed, int32_t *cf) {
    int32_t *Trp, *Tci;
    transpose_pattern(n, Srp, Sci, &Trp, &Tci);
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    for (int32_t i = 0; i < n; ++i) {
        uint64_t deg = (uint64_t)(Trp[i + 1] - Trp[i]);
        key[i] = (deg << 32) | (splitmix64_at(seed, (uint64_t)i) >> 32);
        int isolated = (Srp[i + 1] == Srp[i]) && (Trp[i + 1] == Trp[i]);
        cf[i] = isolated ? 2 : 0;
    }
    uint8_t *newc = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    for (;;) {
        int32_t undecided = 0;
        for (int32_t i = 0; i < n; ++i) undecided += (cf[i] == 0);
        if (!undecided) break;
        /* 1. undecided local maxima over undecided strong neighbours (S_i and S^T_i) */
        for (int32_t i = 0; i < n; ++i) {
            newc[i] = 0;
            if (cf[i] != 0) continue;
            int ok = 1;
            for (int32_t k = Srp[i]; k < Srp[i + 1] && ok; ++k) {
                int32_t j = Sci[k];
                if (cf[j] == 0 && !beats(key[i], i, key[j], j)) ok = 0;
            }
            for (int32_t k = Trp[i]; k < Trp[i + 1] && ok; ++k) {
                int32_t j = Tci[k];
                if (cf[j] == 0 && !beats(key[i], i, key[j], j)) ok = 0;
            }
            newc[i] = (uint8_t)ok;
        }
        for (int32_t i = 0; i < n; ++i)
            if (newc[i]) cf[i] = 1;
        /* 2. undecided points that strongly depend on a C point become F */
        for (int32_t i = 0; i < n; ++i) {
            if (cf[i] != 0) continue;
            for (int32_t k = Srp[i]; k < Srp[i + 1]; ++k)
                if (cf[Sci[k]] == 1) { cf[i] = 2; break; }
        }
    }
    free(newc); free(key); free(Trp); free(Tci);
}

/* Direct interpolation (Stueben): for an F point i with strong C neighbours C_i,
 *   w_ij = -alpha a_ij / (a_ii + sum_{k != i, a_ik > 0} a_ik),
 *   alpha = (sum_{k != i, a_ik < 0} a_ik) / (sum_{k in C_i} a_ik).
 * Strong neighbours are negative entries, so positive couplings are lumped into the diagonal. */
static void direct_interp(const csr *A, const int32_t *Srp, const int32_t *Sci, const int32_t *cf, csr *P,
                          int32_t *nc_out) {
    int32_t n = A->n;
    int32_t *cidx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t nc = 0;
    for (int32_t i = 0; i < n; ++i) cidx[i] = (cf[i] == 1) ? nc++ : -1;
    /* count */
    int32_t *cnt = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    for (int32_t i = 0; i < n; ++i) {
        if (cf[i] == 1) { cnt[i + 1] = 1; continue; }
        int32_t c = 0;
        for (int32_t k = Srp[i]; k < Srp[i + 1]; ++k) c += (cf[Sci[k]] == 1);
        cnt[i + 1] = c;
    }
    for (int32_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    csr_alloc(P, n, cnt[n]);
    memcpy(P->rp, cnt, sizeof(int32_t) * ((size_t)n + 1));
    for (int32_t i = 0; i < n; ++i) {
        int32_t o = P->rp[i];
        if (cf[i] == 1) { P->ci[o] = cidx[i]; P->v[o] = 1.0; continue; }
        if (P->rp[i + 1] == o) continue;
        double aii = 0.0, sneg = 0.0, spos = 0.0, sc = 0.0;
        for (int32_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
            int32_t j = A->ci[k];
            double a = A->v[k];
            if (j == i) aii += a;
            else if (a < 0.0) sneg += a;
            else if (a > 0.0) spos += a;
        }
        /* strong C neighbours in ascending column order (S rows are in A's column order) */
        for (int32_t k = Srp[i]; k < Srp[i + 1]; ++k) {
            int32_t j = Sci[k];
            if (cf[j] != 1) continue;
            for (int32_t q = A->rp[i]; q < A->rp[i + 1]; ++q)
                if (A->ci[q] == j) { sc += A->v[q]; break; }
        }
        double d = aii + spos;
        double alpha = sneg / sc;
        for (int32_t k = Srp[i]; k < Srp[i + 1]; ++k) {
            int32_t j = Sci[k];
            if (cf[j] != 1) continue;
            double a = 0.0;
            for (int32_t q = A->rp[i]; q < A->rp[i + 1]; ++q)
                if (A->ci[q] == j) { a = A->v[q]; break; }
            P->ci[o] = cidx[j];
            P->v[o] = -alpha * a / d;
            ++o;
        }
    }
    free(cnt); free(cidx);
    *nc_out = nc;
}

static void csr_transpose(const csr *A, int32_t ncols, csr *T) {
    csr_alloc(T, ncols, A->nnz);
    for (int32_t k = 0; k < A->nnz; ++k) T->rp[A->ci[k] + 1]++;
    for (int32_t i = 0; i < ncols; ++i) T->rp[i + 1] += T->rp[i];
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * ((size_t)ncols + 1));
    memcpy(pos, T->rp, sizeof(int32_t) * ((size_t)ncols + 1));
    for (int32_t i = 0; i < A->n; ++i)
        for (int32_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
            int32_t p = pos[A->ci[k]]++;
            T->ci[p] = i;
            T->v[p] = A->v[k];
        }
    free(pos);
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* C = A B (ncols of B = ncb).  Every output entry is accumulated in the order of the inner index
 * (ascending column of A's row, then B's row order), starting from 0.0; output columns ascending. */
static void spgemm(const csr *A, const csr *B, int32_t ncb, csr *C) {
    int32_t n = A->n;
    double *acc = (double *)calloc((size_t)(ncb > 0 ? ncb : 1), sizeof(double));
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ncb > 0 ? ncb : 1));
    for (int32_t j = 0; j < ncb; ++j) mark[j] = -1;
    int32_t *list = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ncb > 0 ? ncb : 1));
    int32_t cap = A->nnz + 16, nnz = 0;
    int32_t *ci = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    double *v = (double *)malloc(sizeof(double) * (size_t)cap);
    int32_t *rp = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    for (int32_t i = 0; i < n; ++i) {
        int32_t len = 0;
        for (int32_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
            int32_t l = A->ci[k];
            double a = A->v[k];
            for (int32_t q = B->rp[l]; q < B->rp[l + 1]; ++q) {
                int32_t j = B->ci[q];
                if (mark[j] != i) { mark[j] = i; acc[j] = 0.0; list[len++] = j; }
                acc[j] = acc[j] + a * B->v[q];
            }
        }
        qsort(list, (size_t)len, sizeof(int32_t), cmp_i32);
        if (nnz + len > cap) {
            while (nnz + len > cap) cap *= 2;
            ci = (int32_t *)realloc(ci, sizeof(int32_t) * (size_t)cap);
            v = (double *)realloc(v, sizeof(double) * (size_t)cap);
        }
        for (int32_t t = 0; t < len; ++t) { ci[nnz] = list[t]; v[nnz] = acc[list[t]]; ++nnz; }
        rp[i + 1] = nnz;
    }
    free(acc); free(mark); free(list);
    C->n = n; C->nnz = nnz; C->rp = rp; C->ci = ci; C->v = v;
}

static void smoother_diag(const csr *A, int smoother, double omega, double *dinv) {
    for (int32_t i = 0; i < A->n; ++i) {
        double d = 0.0;
        if (smoother == OR_L1) {
            for (int32_t k = A->rp[i]; k < A->rp[i + 1]; ++k) d += fabs(A->v[k]);
            dinv[i] = 1.0 / d;
        } else {
            for (int32_t k = A->rp[i]; k < A->rp[i + 1]; ++k)
                if (A->ci[k] == i) d += A->v[k];
            dinv[i] = omega / d;
        }
    }
}

/* dense LU with partial pivoting, in place, row-major; returns 0 or -1 if singular */
static int dense_lu(int32_t n, double *a, int32_t *piv) {
    for (int32_t k = 0; k < n; ++k) {
        int32_t p = k;
        double m = fabs(a[(size_t)k * n + k]);
        for (int32_t i = k + 1; i < n; ++i)
            if (fabs(a[(size_t)i * n + k]) > m) { m = fabs(a[(size_t)i * n + k]); p = i; }
        piv[k] = p;
        if (m == 0.0) return -1;
        if (p != k)
            for (int32_t j = 0; j < n; ++j) {
                double t = a[(size_t)k * n + j]; a[(size_t)k * n + j] = a[(size_t)p * n + j]; a[(size_t)p * n + j] = t;
            }
        for (int32_t i = k + 1; i < n; ++i) {
            double l = a[(size_t)i * n + k] / a[(size_t)k * n + k];
            a[(size_t)i * n + k] = l;
            for (int32_t j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
        }
    }
    return 0;
}
static void dense_lu_solve(int32_t n, const double *lu, const int32_t *piv, const double *b, double *x) {
    memcpy(x, b, sizeof(double) * (size_t)n);
    for (int32_t k = 0; k < n; ++k) {
        int32_t p = piv[k];
        if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; }
    }
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < i; ++j) x[i] -= lu[(size_t)i * n + j] * x[j];
    for (int32_t i = n - 1; i >= 0; --i) {
        for (int32_t j = i + 1; j < n; ++j) x[i] -= lu[(size_t)i * n + j] * x[j];
        x[i] /= lu[(size_t)i * n + i];
    }
}

static void csr_copy(const csr *A, csr *B) {
    csr_alloc(B, A->n, A->nnz);
    memcpy(B->rp, A->rp, sizeof(int32_t) * ((size_t)A->n + 1));
    memcpy(B->ci, A->ci, sizeof(int32_t) * (size_t)A->nnz);
    memcpy(B->v, A->v, sizeof(double) * (size_t)A->nnz);
}

static int amg_setup(amg *h, const csr *A0, const or_opts *o) {
    memset(h, 0, sizeof(*h));
    csr_copy(A0, &h->L[0].A);
    int l = 0;
    int maxl = o->max_levels < 1 ? 1 : (o->max_levels > 32 ? 32 : o->max_levels);
    for (;;) {
        amg_level *L = &h->L[l];
        int32_t n = L->A.n;
        L->dinv = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        smoother_diag(&L->A, o->smoother, o->omega, L->dinv);
        L->r = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
        L->x = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
        L->b = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
        if (l + 1 >= maxl || n <= o->n_coarse) break;
        int32_t *Srp, *Sci;
        strength(&L->A, o->theta, &Srp, &Sci);
        L->cf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        pmis(n, Srp, Sci, (uint64_t)o->seed + (uint64_t)l, L->cf);
        int32_t nc;
        direct_interp(&L->A, Srp, Sci, L->cf, &L->P, &nc);
        free(Srp); free(Sci);
        if (nc == 0 || nc >= n) { /* no coarsening possible: this level is the coarsest */
            csr_free(&L->P); free(L->cf); L->cf = NULL;
            break;
        }
        csr_transpose(&L->P, nc, &L->PT);
        csr AP;
        spgemm(&L->A, &L->P, nc, &AP);
        spgemm(&L->PT, &AP, nc, &h->L[l + 1].A);
        csr_free(&AP);
        ++l;
    }
    h->nlev = l + 1;
    amg_level *C = &h->L[l];
    int32_t n = C->A.n;
    if (n <= o->dense_max) {
        h->dense = 1;
        h->lu = (double *)calloc((size_t)n * n + 1, sizeof(double));
        h->piv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
        for (int32_t i = 0; i < n; ++i)
            for (int32_t k = C->A.rp[i]; k < C->A.rp[i + 1]; ++k) h->lu[(size_t)i * n + C->A.ci[k]] += C->A.v[k];
        if (dense_lu(n, h->lu, h->piv) != 0) return -6;
    }
    return 0;
}

static void amg_free(amg *h) {
    for (int l = 0; l < h->nlev; ++l) {
        amg_level *L = &h->L[l];
        csr_free(&L->A); csr_free(&L->P); csr_free(&L->PT);
        free(L->dinv); free(L->cf); free(L->r); free(L->x); free(L->b);
    }
    free(h->lu); free(h->piv);
    memset(h, 0, sizeof(*h));
}

/* The diagonal block of rows and columns [r0, r1) of A, re-indexed from 0. */
static void extract_block(const csr *A, int32_t r0, int32_t r1, csr *B) {
    int32_t nnz = 0;
    for (int32_t i = r0; i < r1; ++i)
        for (int32_t k = A->rp[i]; k < A->rp[i + 1]; ++k) nnz += (A->ci[k] >= r0 && A->ci[k] < r1);
    csr_alloc(B, r1 - r0, nnz);
    int32_t o = 0;
    for (int32_t i = r0; i < r1; ++i) {
        for (int32_t k = A->rp[i]; k < A->rp[i + 1]; ++k)
            if (A->ci[k] >= r0 && A->ci[k] < r1) { B->ci[o] = A->ci[k] - r0; B->v[o] = A->v[k]; ++o; }
        B->rp[i - r0 + 1] = o;
    }
}

/* Unknown-based AMG (Sec. 3.4) on A_00 in unknown-wise order: rows [0, np) are the pressure
 * unknowns, rows [np, n) the temperature unknowns.  On every level, classical coarsening (strength,
 * PMIS) and direct interpolation are applied to each diagonal block on its own (the pressure block
 * and the temperature block, with PMIS weights indexed within the block), P = blockdiag(P_p, P_T)
 * with the coarse pressure points first, and the coarse operator is the Galerkin product of the
 * whole coupled level matrix, A_c = P^T (A P), so the coupling blocks stay in the coarse-grid
 * correction.  The smoother and the coarsest solve act on the whole level matrix.  Coarsening stops
 * as in amg_setup (n <= n_coarse, max_levels, or no coarsening possible in either block). */
static int uamg_setup(amg *h, const csr *A0, int32_t np0, const or_opts *o) {
    memset(h, 0, sizeof(*h));
    csr_copy(A0, &h->L[0].A);
    int l = 0;
    int32_t np = np0;
    int maxl = o->max_levels < 1 ? 1 : (o->max_levels > 32 ? 32 : o->max_levels);
    for (;;) {
        amg_level *L = &h->L[l];
        int32_t n = L->A.n;
        L->dinv = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        smoother_diag(&L->A, o->smoother, o->omega, L->dinv);
        L->r = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
        L->x = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
        L->b = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
        if (l + 1 >= maxl || n <= o->n_coarse) break;
        /* each unknown's diagonal block: strength, PMIS, direct interpolation */
        csr blk[2], Pb[2];
        int32_t nc[2], r0[2] = {0, np}, r1[2] = {np, n};
        int32_t *cfb[2];
        for (int u = 0; u < 2; ++u) {
            extract_block(&L->A, r0[u], r1[u], &blk[u]);
            int32_t *Srp, *Sci;
            strength(&blk[u], o->theta, &Srp, &Sci);
            cfb[u] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(blk[u].n > 0 ? blk[u].n : 1));
            pmis(blk[u].n, Srp, Sci, (uint64_t)o->seed + (uint64_t)l, cfb[u]);
            direct_interp(&blk[u], Srp, Sci, cfb[u], &Pb[u], &nc[u]);
            free(Srp); free(Sci);
        }
        int32_t ncs = nc[0] + nc[1];
        if (ncs == 0 || ncs >= n) { /* no coarsening possible: this level is the coarsest */
            for (int u = 0; u < 2; ++u) { csr_free(&blk[u]); csr_free(&Pb[u]); free(cfb[u]); }
            break;
        }
        /* P = blockdiag(P_p, P_T): temperature columns after the nc[0] pressure columns */
        csr_alloc(&L->P, n, Pb[0].nnz + Pb[1].nnz);
        L->cf = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        int32_t o2 = 0;
        for (int u = 0; u < 2; ++u)
            for (int32_t i = 0; i < Pb[u].n; ++i) {
                L->cf[r0[u] + i] = cfb[u][i];
                for (int32_t k = Pb[u].rp[i]; k < Pb[u].rp[i + 1]; ++k) {
                    L->P.ci[o2] = Pb[u].ci[k] + (u ? nc[0] : 0);
                    L->P.v[o2] = Pb[u].v[k];
                    ++o2;
                }
                L->P.rp[r0[u] + i + 1] = o2;
            }
        for (int u = 0; u < 2; ++u) { csr_free(&blk[u]); csr_free(&Pb[u]); free(cfb[u]); }
        csr_transpose(&L->P, ncs, &L->PT);
        csr AP;
        spgemm(&L->A, &L->P, ncs, &AP);
        spgemm(&L->PT, &AP, ncs, &h->L[l + 1].A);
        csr_free(&AP);
        np = nc[0];
        ++l;
    }
    h->nlev = l + 1;
    amg_level *C = &h->L[l];
    int32_t n = C->A.n;
    if (n <= o->dense_max) {
        h->dense = 1;
        h->lu = (double *)calloc((size_t)n * n + 1, sizeof(double));
        h->piv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
        for (int32_t i = 0; i < n; ++i)
            for (int32_t k = C->A.rp[i]; k < C->A.rp[i + 1]; ++k) h->lu[(size_t)i * n + C->A.ci[k]] += C->A.v[k];
        if (dense_lu(n, h->lu, h->piv) != 0) return -6;
    }
    return 0;
}

/* One V(1,1)-cycle with zero initial guess: x ~= A_l^{-1} b. */
static void vcycle(amg *h, int l, const double *b, double *x) {
    amg_level *L = &h->L[l];
    int32_t n = L->A.n;
    if (l == h->nlev - 1) {
        if (h->dense) { dense_lu_solve(n, h->lu, h->piv, b, x); return; }
        for (int32_t i = 0; i < n; ++i) x[i] = L->dinv[i] * b[i];
        spmv(&L->A, x, L->r);
        for (int32_t i = 0; i < n; ++i) x[i] = x[i] + L->dinv[i] * (b[i] - L->r[i]);
        return;
    }
    amg_level *Cl = &h->L[l + 1];
    /* pre-smoothing from zero: x = D^{-1} b */
    for (int32_t i = 0; i < n; ++i) x[i] = L->dinv[i] * b[i];
    /* residual r = b - A x, restriction b_c = P^T r */
    spmv(&L->A, x, L->r);
    for (int32_t i = 0; i < n; ++i) L->r[i] = b[i] - L->r[i];
    spmv(&L->PT, L->r, Cl->b);
    vcycle(h, l + 1, Cl->b, Cl->x);
    /* prolongation x += P x_c */
    spmv(&L->P, Cl->x, L->r);
    for (int32_t i = 0; i < n; ++i) x[i] += L->r[i];
    /* post-smoothing x = x + D^{-1}(b - A x) */
    spmv(&L->A, x, L->r);
    for (int32_t i = 0; i < n; ++i) L->r[i] = x[i] + L->dinv[i] * (b[i] - L->r[i]);
    memcpy(x, L->r, sizeof(double) * (size_t)n);
}

/* ------------------------------------------------------------------------------------------ */
/* ILU(0) on the interleaved scalar CSR (IKJ form, no pivoting)                                 */
typedef struct {
    csr LU;        /* L (unit, strictly lower) and U (upper incl. diagonal) in A's pattern */
    int32_t *diag; /* position of the diagonal in each row */
} ilu0;

static int ilu0_factor(const csr *A, ilu0 *f) {
    csr_copy(A, &f->LU);
    int32_t n = A->n;
    f->diag = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int32_t j = 0; j < n; ++j) pos[j] = -1;
    csr *M = &f->LU;
    for (int32_t i = 0; i < n; ++i) {
        f->diag[i] = -1;
        for (int32_t k = M->rp[i]; k < M->rp[i + 1]; ++k)
            if (M->ci[k] == i) f->diag[i] = k;
        if (f->diag[i] < 0) { free(pos); return -1; }
    }
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t k = M->rp[i]; k < M->rp[i + 1]; ++k) pos[M->ci[k]] = k;
        for (int32_t k = M->rp[i]; k < M->rp[i + 1]; ++k) {
            int32_t c = M->ci[k];
            if (c >= i) break;
            double piv = M->v[f->diag[c]];
            if (piv == 0.0) { free(pos); return -6; }
            M->v[k] = M->v[k] / piv;
            double lik = M->v[k];
            for (int32_t q = f->diag[c] + 1; q < M->rp[c + 1]; ++q) {
                int32_t p = pos[M->ci[q]];
                if (p >= 0) M->v[p] = M->v[p] - lik * M->v[q];
            }
        }
        for (int32_t k = M->rp[i]; k < M->rp[i + 1]; ++k) pos[M->ci[k]] = -1;
        if (M->v[f->diag[i]] == 0.0) { free(pos); return -6; }
    }
    free(pos);
    return 0;
}

/* The ILU(1) pattern: row i keeps its own entries and gains, for every entry k < i of its row,
 * the entries j > k of row k (a fill entry has level lev(i,k) + lev(k,j) + 1, which is at most 1
 * only when both are original entries, so the original pattern alone decides).  F holds A's
 * values, zero at the fill; ILU on this pattern (ilu0_factor) is ILU(1) of A. */
static void ilu1_pattern(const csr *A, csr *F) {
    int32_t n = A->n;
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *list = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int32_t j = 0; j < n; ++j) mark[j] = -1;
    int32_t cap = 2 * A->nnz + 16, nnz = 0;
    F->n = n;
    F->rp = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    F->ci = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    F->v = (double *)malloc(sizeof(double) * (size_t)cap);
    for (int32_t i = 0; i < n; ++i) {
        int32_t len = 0;
        for (int32_t k = A->rp[i]; k < A->rp[i + 1]; ++k) { mark[A->ci[k]] = i; list[len++] = A->ci[k]; }
        for (int32_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
            int32_t kc = A->ci[k];
            if (kc >= i) break;
            for (int32_t q = A->rp[kc]; q < A->rp[kc + 1]; ++q) {
                int32_t j = A->ci[q];
                if (j > kc && mark[j] != i) { mark[j] = i; list[len++] = j; }
            }
        }
        qsort(list, (size_t)len, sizeof(int32_t), cmp_i32);
        if (nnz + len > cap) {
            while (nnz + len > cap) cap *= 2;
            F->ci = (int32_t *)realloc(F->ci, sizeof(int32_t) * (size_t)cap);
            F->v = (double *)realloc(F->v, sizeof(double) * (size_t)cap);
        }
        int32_t a = A->rp[i];
        for (int32_t t = 0; t < len; ++t) {
            F->ci[nnz] = list[t];
            F->v[nnz] = (a < A->rp[i + 1] && A->ci[a] == list[t]) ? A->v[a++] : 0.0;
            ++nnz;
        }
        F->rp[i + 1] = nnz;
    }
    F->nnz = nnz;
    free(mark); free(list);
}

/* Block Jacobi (Sec. 4: in parallel, ILU(k) on each block of the domain's partition): the entries
 * of A whose row and column cells (scalar index / b) lie in the same part.  ILU(0) on this pattern
 * factors every part on its own. */
static void partition_pattern(const csr *A, int32_t b, const int32_t *part, csr *F) {
    int32_t n = A->n;
    F->n = n;
    F->rp = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    F->ci = (int32_t *)malloc(sizeof(int32_t) * (size_t)(A->nnz > 0 ? A->nnz : 1));
    F->v = (double *)malloc(sizeof(double) * (size_t)(A->nnz > 0 ? A->nnz : 1));
    int32_t nnz = 0;
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t k = A->rp[i]; k < A->rp[i + 1]; ++k)
            if (part[A->ci[k] / b] == part[i / b]) {
                F->ci[nnz] = A->ci[k];
                F->v[nnz] = A->v[k];
                ++nnz;
            }
        F->rp[i + 1] = nnz;
    }
    F->nnz = nnz;
}

static void ilu0_solve(const ilu0 *f, const double *r, double *z) {
    const csr *M = &f->LU;
    int32_t n = M->n;
    for (int32_t i = 0; i < n; ++i) {
        double s = r[i];
        for (int32_t k = M->rp[i]; k < f->diag[i]; ++k) s -= M->v[k] * z[M->ci[k]];
        z[i] = s;
    }
    for (int32_t i = n - 1; i >= 0; --i) {
        double s = z[i];
        for (int32_t k = f->diag[i] + 1; k < M->rp[i + 1]; ++k) s -= M->v[k] * z[M->ci[k]];
        z[i] = s / M->v[f->diag[i]];
    }
}

/* ------------------------------------------------------------------------------------------ */
/* the solver context                                                                           */
typedef struct {
    or_opts o;
    int32_t n, b, ps, ts;
    csr A;             /* decoupled A' (interleaved scalar CSR) */
    csr Alow;          /* mixed precision: A' with FP32-rounded values for the stage-1 residual */
    double *W;         /* [n, b, b] row weights (identity if none was given) */
    csr App, ApT, ATp, St;
    amg hp, hT;
    csr A00;           /* uAMG: A_00 in unknown-wise order [p; T] */
    double *Ddec;      /* decoupling: D_i of every cell, [n][2][b] (rows p, T; columns by slot, zero
                          outside the secondary slots) */
    amg hU;
    double *b00, *x00;
    ilu0 ilu;
    int32_t *cperm;    /* multicolour ILU: new cell index -> original cell (NULL: natural) */
    csr Aperm;         /* A' with cells permuted (multicolour ILU only) */
    double *rp_tmp, *zp_tmp;
    /* work */
    double *bp, *bT, *xp, *dT, *dp, *t1, *x1, *b1;
    int status;
} or_ctx;

/* Expand BSR (row-major b x b blocks) to the interleaved scalar CSR, applying W if given:
 * block row i of A' is W_i times block row i of A (Sec. 2.2.2 eq. weighted, Sec. 3.5 eq. scaling). */
static void bsr_to_csr_weighted(int32_t n, int32_t b, const int32_t *rp, const int32_t *ci, const double *vals,
                                const double *W, csr *A) {
    int64_t nnzb = rp[n];
    csr_alloc(A, n * b, (int32_t)(nnzb * b * b));
    int32_t o = 0;
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t r = 0; r < b; ++r) {
            for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
                const double *blk = vals + (int64_t)k * b * b;
                for (int32_t c = 0; c < b; ++c) {
                    double s;
                    if (W) {
                        s = 0.0;
                        for (int32_t t = 0; t < b; ++t) s += W[(int64_t)i * b * b + r * b + t] * blk[t * b + c];
                    } else {
                        s = blk[r * b + c];
                    }
                    A->ci[o] = ci[k] * b + c;
                    A->v[o] = s;
                    ++o;
                }
            }
            A->rp[i * b + r + 1] = o;
        }
    }
}

/* Scalar block (u, w) of A': entries A'(i*b+u, j*b+w) on the cell pattern (Sec. 3.2 eq. A00). */
static void extract_field(const or_ctx *c, const int32_t *rp, const int32_t *ci, int u, int w, csr *F) {
    int32_t n = c->n, b = c->b;
    csr_alloc(F, n, rp[n]);
    memcpy(F->rp, rp, sizeof(int32_t) * ((size_t)n + 1));
    memcpy(F->ci, ci, sizeof(int32_t) * (size_t)rp[n]);
    for (int32_t i = 0; i < n; ++i) {
        int32_t row = i * b + u;
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
            /* in the interleaved CSR, block k of cell row i occupies b consecutive entries */
            int32_t base = c->A.rp[row] + (k - rp[i]) * b;
            F->v[k] = c->A.v[base + w];
        }
    }
}

/* Rounding to the storage formats of the mixed-precision form.  FP32: IEEE round to nearest
 * (the C conversion).  BF16: the FP32 value rounded to 8 significant bits, round to nearest, ties
 * to even (keep the top 16 bits of the binary32 encoding). */
static double round_fp32(double x) { return (double)(float)x; }
static double round_bf16(double x) {
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return (double)f;   /* inf / nan unchanged */
    u += 0x7FFFu + ((u >> 16) & 1u);
    u &= 0xFFFF0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}
static void round_array(double *v, int64_t n, int bf16) {
    for (int64_t i = 0; i < n; ++i) v[i] = bf16 ? round_bf16(v[i]) : round_fp32(v[i]);
}
/* levels 0 and 1 in FP32, levels >= 2 in BF16 (matrix and transfer values); the smoother
 * diagonal in FP32; the coarsest dense factorisation stays FP64 */
static void round_hierarchy(amg *h) {
    for (int l = 0; l < h->nlev; ++l) {
        amg_level *L = &h->L[l];
        int bf = l >= 2;
        round_array(L->A.v, L->A.nnz, bf);
        if (L->P.rp) round_array(L->P.v, L->P.nnz, bf);
        if (L->PT.rp) round_array(L->PT.v, L->PT.nnz, bf);
        round_array(L->dinv, L->A.n, 0);
    }
}
double or_round_bf16(double x) { return round_bf16(x); }

/* Greedy distance-1 colouring of the cell graph in natural order (each cell takes the smallest
 * colour not used by its lower-index neighbours), then cells sorted by (colour, index).  Returns
 * the order: new index -> original cell.  On a 7-point Cartesian grid this is red-black. */
static int32_t *multicolour_order(int32_t n, const int32_t *rp, const int32_t *ci) {
    int32_t *color = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t ncol = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t c = 0;
        for (;;) {
            int used = 0;
            for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
                if (ci[k] < i && color[ci[k]] == c) { used = 1; break; }
            if (!used) break;
            ++c;
        }
        color[i] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t o = 0;
    for (int32_t c = 0; c < ncol; ++c)
        for (int32_t i = 0; i < n; ++i)
            if (color[i] == c) order[o++] = i;
    free(color);
    return order;
}

/* P A P^T for a cell permutation (order: new -> original) of the interleaved scalar CSR:
 * unknown u of new cell I is row I*b + u; columns renumbered likewise and sorted. */
static int cmp_pair(const void *a, const void *b) {
    int32_t x = ((const int32_t *)a)[0], y = ((const int32_t *)b)[0];
    return (x > y) - (x < y);
}
static void permute_cells(const csr *A, int32_t b, const int32_t *order, csr *P) {
    int32_t n = A->n / b;
    int32_t *inv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int32_t I = 0; I < n; ++I) inv[order[I]] = I;
    csr_alloc(P, A->n, A->nnz);
    int32_t o = 0;
    int32_t *pairs = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(A->n > 0 ? A->n : 1));
    for (int32_t I = 0; I < n; ++I)
        for (int32_t u = 0; u < b; ++u) {
            int32_t row = order[I] * b + u, len = A->rp[row + 1] - A->rp[row];
            for (int32_t t = 0; t < len; ++t) {
                int32_t c = A->ci[A->rp[row] + t];
                pairs[2 * t] = inv[c / b] * b + c % b;
                pairs[2 * t + 1] = A->rp[row] + t;
            }
            qsort(pairs, (size_t)len, 2 * sizeof(int32_t), cmp_pair);
            for (int32_t t = 0; t < len; ++t) {
                P->ci[o] = pairs[2 * t];
                P->v[o] = A->v[pairs[2 * t + 1]];
                ++o;
            }
            P->rp[I * b + u + 1] = o;
        }
    free(pairs);
    free(inv);
}

/* z = (LU)^{-1} r for the factors of the (possibly cell-permuted) matrix */
/* entry (r, c) of block k (block row i) of the interleaved scalar CSR A' */
static double blk_at(const or_ctx *c, const int32_t *rp, int32_t i, int32_t k, int r, int col) {
    int32_t b = c->b;
    return c->A.v[c->A.rp[i * b + r] + (k - rp[i]) * b + col];
}

/* the primary slots of the decoupled first stage: {p} for CPR, {p, T} for the p-T first stages */
static int primary_slots(const or_ctx *c, int *prim) {
    prim[0] = c->ps;
    if (c->o.stage1 == OR_CPR) return 1;
    prim[1] = c->ts;
    return 2;
}

/* in-place inverse of an m x m row-major matrix by Gauss-Jordan elimination with partial pivoting
 * (largest |y_rk| among the remaining rows, lowest row on ties; the pivot row times 1 / pivot;
 * every other row minus its multiple of the pivot row); returns -1 if singular */
static int small_inverse(int m, double *y) {
    double a[3][6];
    for (int r = 0; r < m; ++r)
        for (int q = 0; q < 2 * m; ++q) a[r][q] = q < m ? y[r * m + q] : (q - m == r ? 1.0 : 0.0);
    for (int k = 0; k < m; ++k) {
        int p = k;
        for (int r = k + 1; r < m; ++r)
            if (fabs(a[r][k]) > fabs(a[p][k])) p = r;
        if (a[p][k] == 0.0) return -1;
        if (p != k)
            for (int q = 0; q < 2 * m; ++q) { double t = a[k][q]; a[k][q] = a[p][q]; a[p][q] = t; }
        double inv = 1.0 / a[k][k];
        for (int q = 0; q < 2 * m; ++q) a[k][q] = a[k][q] * inv;
        for (int r = 0; r < m; ++r) {
            if (r == k) continue;
            double f = a[r][k];
            for (int q = 0; q < 2 * m; ++q) a[r][q] = a[r][q] - f * a[k][q];
        }
    }
    for (int r = 0; r < m; ++r)
        for (int q = 0; q < m; ++q) y[r * m + q] = a[r][m + q];
    return 0;
}

/* Decoupling operator G = [I -D; 0 I] (Sec. 3.1 for CPR, extended to the p-T system in Sec. 3.2):
 * D_i = X_i Y_i^{-1} per cell, with X_i from the primary rows and secondary columns and Y_i from
 * the secondary rows and columns of A'.  Quasi-IMPES: the cell's diagonal block (diag);
 * True-IMPES: the sum of the blocks in the cell's block column (colsum), over the block rows j
 * ascending.  D_i[r][t] = sum over u ascending of X_i[r][u] Yinv_i[u][t]. */
static int compute_decoupling(or_ctx *c, const int32_t *rp, const int32_t *ci) {
    int32_t n = c->n, b = c->b;
    int prim[2], sec[4], np_ = primary_slots(c, prim), ns = 0;
    for (int q = 0; q < b; ++q) {
        int is_p = 0;
        for (int t = 0; t < np_; ++t) is_p |= (prim[t] == q);
        if (!is_p) sec[ns++] = q;
    }
    c->Ddec = (double *)calloc((size_t)n * 2 * b, sizeof(double));
    for (int32_t i = 0; i < n; ++i) {
        double X[2][3] = {{0}}, Y[9] = {0};
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
            int32_t j = ci[k];
            if (c->o.decouple == 1) {          /* QI: the diagonal block of row i */
                if (j != i) continue;
                for (int r = 0; r < np_; ++r)
                    for (int t = 0; t < ns; ++t) X[r][t] = blk_at(c, rp, i, k, prim[r], sec[t]);
                for (int r = 0; r < ns; ++r)
                    for (int t = 0; t < ns; ++t) Y[r * ns + t] = blk_at(c, rp, i, k, sec[r], sec[t]);
            } else {                           /* TI: block (j, i) of every row j with one */
                int32_t kk = -1;
                for (int32_t q = rp[j]; q < rp[j + 1]; ++q)
                    if (ci[q] == i) { kk = q; break; }
                if (kk < 0) return -1;         /* the pattern must be structurally symmetric */
                for (int r = 0; r < np_; ++r)
                    for (int t = 0; t < ns; ++t) X[r][t] = X[r][t] + blk_at(c, rp, j, kk, prim[r], sec[t]);
                for (int r = 0; r < ns; ++r)
                    for (int t = 0; t < ns; ++t) Y[r * ns + t] = Y[r * ns + t] + blk_at(c, rp, j, kk, sec[r], sec[t]);
            }
        }
        if (small_inverse(ns, Y) != 0) return -6;
        for (int r = 0; r < np_; ++r)
            for (int t = 0; t < ns; ++t) {
                double d = 0.0;
                for (int u = 0; u < ns; ++u) d = d + X[r][u] * Y[u * ns + t];
                c->Ddec[((size_t)i * 2 + r) * b + sec[t]] = d;
            }
    }
    return 0;
}

/* Field (u, w) of G A' on the cell pattern: entry a(i,u; j,w) - sum_s D_i[u][s] a(i,s; j,w) over the
 * secondary slots s ascending (u a primary slot). */
static void extract_field_g(const or_ctx *c, const int32_t *rp, const int32_t *ci, int u, int w, csr *F) {
    int32_t n = c->n, b = c->b;
    int ru = (u == c->ps) ? 0 : 1;
    csr_alloc(F, n, rp[n]);
    memcpy(F->rp, rp, sizeof(int32_t) * ((size_t)n + 1));
    memcpy(F->ci, ci, sizeof(int32_t) * (size_t)rp[n]);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
            double v = blk_at(c, rp, i, k, u, w);
            for (int s = 0; s < b; ++s) {
                double d = c->Ddec[((size_t)i * 2 + ru) * b + s];
                if (d != 0.0) v = v - d * blk_at(c, rp, i, k, s, w);
            }
            F->v[k] = v;
        }
}

/* A_00 = [A_pp A_pT; A_Tp A_TT] in unknown-wise order (Sec. 3.2 eq. A00): row i < n holds A_pp row
 * i (columns j) then A_pT row i (columns n + j); row n + i holds A_Tp row i then A_TT row i. */
static void assemble_a00(const csr *App, const csr *ApT, const csr *ATp, const csr *ATT, csr *A) {
    int32_t n = App->n;
    csr_alloc(A, 2 * n, App->nnz + ApT->nnz + ATp->nnz + ATT->nnz);
    int32_t o = 0;
    const csr *row_blocks[2][2] = {{App, ApT}, {ATp, ATT}};
    for (int u = 0; u < 2; ++u)
        for (int32_t i = 0; i < n; ++i) {
            for (int w = 0; w < 2; ++w) {
                const csr *F = row_blocks[u][w];
                for (int32_t k = F->rp[i]; k < F->rp[i + 1]; ++k) {
                    A->ci[o] = F->ci[k] + (w ? n : 0);
                    A->v[o] = F->v[k];
                    ++o;
                }
            }
            A->rp[u * n + i + 1] = o;
        }
}

/* S~_diag = A_TT - A_Tp diag(A_pp)^{-1} A_pT (Sec. 3.3.1): the product column-scales A_Tp by
 * 1 / (A_pp)_kk, then multiplies by A_pT (each entry summed over k ascending); the difference is
 * taken on the union pattern, columns ascending. */
static void schur_diag(const or_ctx *c, const int32_t *rp, const int32_t *ci, csr *S) {
    int32_t n = c->n;
    csr ATT, B, C;
    extract_field(c, rp, ci, c->ts, c->ts, &ATT);
    csr_copy(&c->ATp, &B);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = B.rp[i]; k < B.rp[i + 1]; ++k) {
            int32_t j = B.ci[k];
            double d = 0.0;
            for (int32_t q = c->App.rp[j]; q < c->App.rp[j + 1]; ++q)
                if (c->App.ci[q] == j) d = c->App.v[q];
            B.v[k] = B.v[k] * (1.0 / d);
        }
    spgemm(&B, &c->ApT, n, &C);
    csr_alloc(S, n, ATT.nnz + C.nnz);
    int32_t o = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t a = ATT.rp[i], ae = ATT.rp[i + 1], b = C.rp[i], be = C.rp[i + 1];
        while (a < ae || b < be) {
            int32_t ja = a < ae ? ATT.ci[a] : INT32_MAX, jb = b < be ? C.ci[b] : INT32_MAX;
            if (ja == jb) { S->ci[o] = ja; S->v[o] = ATT.v[a] - C.v[b]; ++a; ++b; }
            else if (ja < jb) { S->ci[o] = ja; S->v[o] = ATT.v[a]; ++a; }
            else { S->ci[o] = jb; S->v[o] = -C.v[b]; ++b; }
            ++o;
        }
        S->rp[i + 1] = o;
    }
    S->nnz = o;
    csr_free(&ATT); csr_free(&B); csr_free(&C);
}

static void ilu_apply_ordered(or_ctx *c, const double *r, double *z) {
    if (!c->cperm) { ilu0_solve(&c->ilu, r, z); return; }
    int32_t b = c->b;
    for (int32_t I = 0; I < c->n; ++I)
        for (int32_t u = 0; u < b; ++u) c->rp_tmp[I * b + u] = r[c->cperm[I] * b + u];
    ilu0_solve(&c->ilu, c->rp_tmp, c->zp_tmp);
    for (int32_t I = 0; I < c->n; ++I)
        for (int32_t u = 0; u < b; ++u) z[c->cperm[I] * b + u] = c->zp_tmp[I * b + u];
}

or_ctx *or_create(int32_t n, int32_t b, const int32_t *rp, const int32_t *ci, const double *vals, const double *W,
                  int32_t ps, int32_t ts, const int32_t *st_rp, const int32_t *st_ci, const double *st_v,
                  const or_opts *o) {
    or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
    c->o = *o;
    c->n = n; c->b = b; c->ps = ps; c->ts = ts;
    c->W = (double *)malloc(sizeof(double) * (size_t)n * b * b);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t r = 0; r < b; ++r)
            for (int32_t t = 0; t < b; ++t)
                c->W[(int64_t)i * b * b + r * b + t] = W ? W[(int64_t)i * b * b + r * b + t] : (r == t ? 1.0 : 0.0);
    bsr_to_csr_weighted(n, b, rp, ci, vals, W, &c->A);
    int rc = 0;
    if (o->decouple) rc = compute_decoupling(c, rp, ci);
    if (c->Ddec) {   /* the first stage's fields of G A' (Sec. 3.1, 3.2) */
        extract_field_g(c, rp, ci, ps, ps, &c->App);
        extract_field_g(c, rp, ci, ps, ts, &c->ApT);
        if (o->stage1 == OR_CPR) extract_field(c, rp, ci, ts, ps, &c->ATp);
        else extract_field_g(c, rp, ci, ts, ps, &c->ATp);
    } else {
        extract_field(c, rp, ci, ps, ps, &c->App);
        extract_field(c, rp, ci, ps, ts, &c->ApT);
        extract_field(c, rp, ci, ts, ps, &c->ATp);
    }
    if (st_v && o->schur == OR_SCHUR_GIVEN) {
        csr_alloc(&c->St, n, st_rp[n]);
        memcpy(c->St.rp, st_rp, sizeof(int32_t) * ((size_t)n + 1));
        memcpy(c->St.ci, st_ci, sizeof(int32_t) * (size_t)st_rp[n]);
        memcpy(c->St.v, st_v, sizeof(double) * (size_t)st_rp[n]);
    } else if (o->schur == OR_SCHUR_DIAG) {
        schur_diag(c, rp, ci, &c->St);             /* S~_diag (Sec. 3.3.1) */
    } else {
        extract_field(c, rp, ci, ts, ts, &c->St); /* S~_{A_TT} = A_TT (Sec. 3.3.1) */
    }
    if (rc) { c->status = rc; return c; }
    if (o->stage1 == OR_UAMG) {
        csr ATT;
        if (c->Ddec) extract_field_g(c, rp, ci, ts, ts, &ATT);
        else extract_field(c, rp, ci, ts, ts, &ATT);
        assemble_a00(&c->App, &c->ApT, &c->ATp, &ATT, &c->A00);
        csr_free(&ATT);
        rc = uamg_setup(&c->hU, &c->A00, n, o);
    } else {
        if (o->stage1 != OR_NONE1) rc = amg_setup(&c->hp, &c->App, o);
        if (!rc && o->stage1 != OR_NONE1 && o->stage1 != OR_CPR) rc = amg_setup(&c->hT, &c->St, o);
    }
    if (!rc && o->stage2 == OR_ILU0) {
        const csr *M = &c->A;
        if (o->ilu_order == 1) {
            c->cperm = multicolour_order(n, rp, ci);
            permute_cells(&c->A, b, c->cperm, &c->Aperm);
            c->rp_tmp = (double *)calloc((size_t)n * b, sizeof(double));
            c->zp_tmp = (double *)calloc((size_t)n * b, sizeof(double));
            M = &c->Aperm;
        }
        if (o->part && (o->ilu_order != 0 || o->ilu_fill != 0)) {
            rc = 2;   /* block Jacobi: natural order and ILU(0) only */
        } else if (o->part) {     /* block-Jacobi ILU(0) */
            csr F;
            partition_pattern(M, b, o->part, &F);
            rc = ilu0_factor(&F, &c->ilu);
            csr_free(&F);
        } else if (o->ilu_fill == 1) {   /* ILU(1): ILU on the level-1 fill pattern */
            csr F;
            ilu1_pattern(M, &F);
            rc = ilu0_factor(&F, &c->ilu);
            csr_free(&F);
        } else {
            rc = ilu0_factor(M, &c->ilu);
        }
    }
    if (!rc && o->precision == 1) {
        round_hierarchy(&c->hp);
        round_hierarchy(&c->hT);
        round_hierarchy(&c->hU);
        round_array(c->ApT.v, c->ApT.nnz, 0);
        round_array(c->ATp.v, c->ATp.nnz, 0);
        csr_copy(&c->A, &c->Alow);            /* A' for the stage-1 residual, FP32 values */
        round_array(c->Alow.v, c->Alow.nnz, 0);
    }
    c->status = rc;
    size_t nb = (size_t)n * b;
    c->bp = calloc(n, sizeof(double)); c->bT = calloc(n, sizeof(double));
    c->xp = calloc(n, sizeof(double)); c->dT = calloc(n, sizeof(double));
    c->dp = calloc(n, sizeof(double)); c->t1 = calloc(n, sizeof(double));
    c->x1 = calloc(nb, sizeof(double)); c->b1 = calloc(nb, sizeof(double));
    c->b00 = calloc(2 * (size_t)n, sizeof(double)); c->x00 = calloc(2 * (size_t)n, sizeof(double));
    return c;
}

int or_status(const or_ctx *c) { return c->status; }

void or_destroy(or_ctx *c) {
    if (!c) return;
    csr_free(&c->A); csr_free(&c->App); csr_free(&c->ApT); csr_free(&c->ATp); csr_free(&c->St);
    amg_free(&c->hp); amg_free(&c->hT); amg_free(&c->hU); csr_free(&c->A00); free(c->b00); free(c->x00);
    free(c->Ddec);
    csr_free(&c->ilu.LU); free(c->ilu.diag);
    free(c->cperm); csr_free(&c->Aperm); free(c->rp_tmp); free(c->zp_tmp); csr_free(&c->Alow);
    free(c->W); free(c->bp); free(c->bT); free(c->xp); free(c->dT); free(c->dp); free(c->t1);
    free(c->x1); free(c->b1);
    free(c);
}

/* First stage: x1 = M1^{-1} v on the p-T unknowns (zero elsewhere). */
static void stage1(or_ctx *c, const double *v, double *x1) {
    int32_t n = c->n, b = c->b;
    memset(x1, 0, sizeof(double) * (size_t)n * b);
    if (c->o.stage1 == OR_NONE1) return;
    for (int32_t i = 0; i < n; ++i) { c->bp[i] = v[i * b + c->ps]; c->bT[i] = v[i * b + c->ts]; }
    if (c->Ddec)   /* the decoupled right-hand side R G v */
        for (int32_t i = 0; i < n; ++i)
            for (int s = 0; s < b; ++s) {
                double dp = c->Ddec[((size_t)i * 2 + 0) * b + s], dT = c->Ddec[((size_t)i * 2 + 1) * b + s];
                if (dp != 0.0) c->bp[i] = c->bp[i] - dp * v[i * b + s];
                if (dT != 0.0) c->bT[i] = c->bT[i] - dT * v[i * b + s];
            }
    switch (c->o.stage1) {
    case OR_CPTR_FULL: /* Sec. 3.3: the five steps */
        vcycle(&c->hp, 0, c->bp, c->xp);                                         /* 1. A_pp x_p = b_p */
        spmv(&c->ATp, c->xp, c->t1);
        for (int32_t i = 0; i < n; ++i) c->t1[i] = c->bT[i] - c->t1[i];          /* 2. b~_T = b_T - A_Tp x_p */
        vcycle(&c->hT, 0, c->t1, c->dT);                                         /* 3. S~_T d_T = b~_T */
        spmv(&c->ApT, c->dT, c->t1);
        for (int32_t i = 0; i < n; ++i) c->t1[i] = c->bp[i] - c->t1[i];          /* 4. b~_p = b_p - A_pT d_T */
        vcycle(&c->hp, 0, c->t1, c->dp);                                         /* 5. A_pp d_p = b~_p */
        break;
    case OR_CPTR_LOWER: /* right factor of eq. (Aschur) dropped */
        vcycle(&c->hp, 0, c->bp, c->dp);
        spmv(&c->ATp, c->dp, c->t1);
        for (int32_t i = 0; i < n; ++i) c->t1[i] = c->bT[i] - c->t1[i];
        vcycle(&c->hT, 0, c->t1, c->dT);
        break;
    case OR_CPTR_UPPER: /* left factor of eq. (Aschur) dropped */
        vcycle(&c->hT, 0, c->bT, c->dT);
        spmv(&c->ApT, c->dT, c->t1);
        for (int32_t i = 0; i < n; ++i) c->t1[i] = c->bp[i] - c->t1[i];
        vcycle(&c->hp, 0, c->t1, c->dp);
        break;
    case OR_BD: /* block diagonal first stage */
        vcycle(&c->hp, 0, c->bp, c->dp);
        vcycle(&c->hT, 0, c->bT, c->dT);
        break;
    case OR_CPR: /* Sec. 3.1: pressure only */
        vcycle(&c->hp, 0, c->bp, c->dp);
        memset(c->dT, 0, sizeof(double) * (size_t)n);
        break;
    case OR_UAMG: /* Sec. 3.4: one unknown-based V-cycle on A_00 [d_p; d_T] = [b_p; b_T] */
        memcpy(c->b00, c->bp, sizeof(double) * (size_t)n);
        memcpy(c->b00 + n, c->bT, sizeof(double) * (size_t)n);
        vcycle(&c->hU, 0, c->b00, c->x00);
        memcpy(c->dp, c->x00, sizeof(double) * (size_t)n);
        memcpy(c->dT, c->x00 + n, sizeof(double) * (size_t)n);
        break;
    }
    for (int32_t i = 0; i < n; ++i) {
        x1[i * b + c->ps] = c->dp[i];
        if (c->o.stage1 != OR_CPR) x1[i * b + c->ts] = c->dT[i];
    }
}

/* Two-stage preconditioner z = M2^{-1}(v - A' x1) + x1, x1 = M1^{-1} v. */
void or_precond(or_ctx *c, const double *v, double *z) {
    int32_t nb = c->n * c->b;
    stage1(c, v, c->x1);
    spmv(c->Alow.rp ? &c->Alow : &c->A, c->x1, c->b1);
    for (int32_t i = 0; i < nb; ++i) c->b1[i] = v[i] - c->b1[i];
    if (c->o.stage2 == OR_ILU0) ilu_apply_ordered(c, c->b1, z);
    else memcpy(z, c->b1, sizeof(double) * (size_t)nb);
    for (int32_t i = 0; i < nb; ++i) z[i] += c->x1[i];
}

/* b' = W b */
void or_weight_rhs(const or_ctx *c, const double *rhs, double *bw) {
    int32_t b = c->b;
    for (int32_t i = 0; i < c->n; ++i)
        for (int32_t r = 0; r < b; ++r) {
            double s = 0.0;
            for (int32_t t = 0; t < b; ++t) s += c->W[(int64_t)i * b * b + r * b + t] * rhs[(int64_t)i * b + t];
            bw[(int64_t)i * b + r] = s;
        }
}

/* Rows [r0, r1) of A' applied to x (indexed from r0): the rows of one diagonal block. */
static void spmv_rows(const csr *A, int32_t r0, int32_t r1, const double *x, double *y) {
    for (int32_t i = r0; i < r1; ++i) {
        double s = 0.0;
        for (int32_t k = A->rp[i]; k < A->rp[i + 1]; ++k) s += A->v[k] * x[A->ci[k] - r0];
        y[i - r0] = s;
    }
}

/* The preconditioner restricted to rows [r0, r1): v is embedded in a zero vector of the whole
 * system, preconditioned, and the same rows are taken back (for a block-diagonal system this is
 * the preconditioner of the block's own system). */
static void precond_rows(or_ctx *c, int32_t r0, int32_t r1, const double *v, double *z, double *full_in,
                         double *full_out) {
    int32_t nb = c->n * c->b;
    if (r0 == 0 && r1 == nb) { or_precond(c, v, z); return; }
    memset(full_in, 0, sizeof(double) * (size_t)nb);
    memcpy(full_in + r0, v, sizeof(double) * (size_t)(r1 - r0));
    or_precond(c, full_in, full_out);
    memcpy(z, full_out + r0, sizeof(double) * (size_t)(r1 - r0));
}

/* Right-preconditioned flexible GMRES(m) from x = 0 on the diagonal block of cells
 * [cell0, cell0 + ncell) of A' x = W rhs (rhs and x indexed from the block's first row). Returns
 * 0 if converged, 1 if not, -4 on a non-finite value, -1 if the block couples to other cells. */
static int fgmres_block(or_ctx *c, int32_t cell0, int32_t ncell, const double *rhs, double *x, double rtol,
                        or_stats *st) {
    int32_t b = c->b, r0 = cell0 * b, r1 = (cell0 + ncell) * b, nb = r1 - r0, m = c->o.restart;
    for (int32_t i = r0; i < r1; ++i)
        for (int32_t k = c->A.rp[i]; k < c->A.rp[i + 1]; ++k)
            if (c->A.ci[k] < r0 || c->A.ci[k] >= r1) return -1;
    int whole = r0 == 0 && r1 == c->n * b;
    double *full_in = whole ? NULL : (double *)malloc(sizeof(double) * (size_t)c->n * b);
    double *full_out = whole ? NULL : (double *)malloc(sizeof(double) * (size_t)c->n * b);
    double *bw = (double *)malloc(sizeof(double) * (size_t)nb);
    double *V = (double *)malloc(sizeof(double) * (size_t)nb * (m + 1));
    double *Z = (double *)malloc(sizeof(double) * (size_t)nb * m);
    double *w = (double *)malloc(sizeof(double) * (size_t)nb);
    double *H = (double *)calloc((size_t)(m + 1) * m, sizeof(double)); /* H[i*m + j] */
    double *h = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    double *h2 = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    double *cs = (double *)malloc(sizeof(double) * (size_t)m), *sn = (double *)malloc(sizeof(double) * (size_t)m);
    double *g = (double *)malloc(sizeof(double) * (size_t)(m + 1)), *y = (double *)malloc(sizeof(double) * (size_t)m);
    for (int32_t i = cell0; i < cell0 + ncell; ++i) /* b' = W b on the block */
        for (int32_t r = 0; r < b; ++r) {
            double s = 0.0;
            for (int32_t t = 0; t < b; ++t)
                s += c->W[(int64_t)i * b * b + r * b + t] * rhs[(int64_t)(i - cell0) * b + t];
            bw[(int64_t)(i - cell0) * b + r] = s;
        }
    memset(x, 0, sizeof(double) * (size_t)nb);
    double bnorm = sqrt(dot(nb, bw, bw));
    int it = 0, restarts = 0, conv = 0, rc = 1;
    double est = 0.0;
    st->bnorm = bnorm;
    if (bnorm == 0.0) { conv = 1; rc = 0; goto done; }
    for (;;) {
        /* r = b' - A' x */
        spmv_rows(&c->A, r0, r1, x, w);
        for (int32_t i = 0; i < nb; ++i) w[i] = bw[i] - w[i];
        double beta = sqrt(dot(nb, w, w));
        est = beta / bnorm;
        if (!isfinite(beta)) { rc = -4; goto done; }
        if (beta <= rtol * bnorm) { conv = 1; rc = 0; goto done; }
        for (int32_t i = 0; i < nb; ++i) V[i] = w[i] / beta;
        memset(g, 0, sizeof(double) * (size_t)(m + 1));
        g[0] = beta;
        int j, k = 0;
        for (j = 0; j < m && it < c->o.max_it; ++j) {
            double *vj = V + (size_t)j * nb, *zj = Z + (size_t)j * nb;
            precond_rows(c, r0, r1, vj, zj, full_in, full_out);
            spmv_rows(&c->A, r0, r1, zj, w);
            /* CGS2: two passes of classical Gram-Schmidt against v_0..v_j */
            for (int32_t q = 0; q <= j; ++q) h[q] = dot(nb, V + (size_t)q * nb, w);
            for (int32_t q = 0; q <= j; ++q) {
                const double *vq = V + (size_t)q * nb;
                for (int32_t i = 0; i < nb; ++i) w[i] -= h[q] * vq[i];
            }
            for (int32_t q = 0; q <= j; ++q) h2[q] = dot(nb, V + (size_t)q * nb, w);
            for (int32_t q = 0; q <= j; ++q) {
                const double *vq = V + (size_t)q * nb;
                for (int32_t i = 0; i < nb; ++i) w[i] -= h2[q] * vq[i];
            }
            for (int32_t q = 0; q <= j; ++q) H[q * m + j] = h[q] + h2[q];
            double hn = sqrt(dot(nb, w, w));
            H[(j + 1) * m + j] = hn;
            ++it;
            if (!isfinite(hn)) { rc = -4; goto done; }
            if (hn > 0.0)
                for (int32_t i = 0; i < nb; ++i) V[(size_t)(j + 1) * nb + i] = w[i] / hn;
            /* apply the previous rotations to column j, then form the new one */
            for (int32_t q = 0; q < j; ++q) {
                double a = H[q * m + j], bq = H[(q + 1) * m + j];
                H[q * m + j] = cs[q] * a + sn[q] * bq;
                H[(q + 1) * m + j] = -sn[q] * a + cs[q] * bq;
            }
            double a = H[j * m + j], bq = H[(j + 1) * m + j];
            double den = sqrt(a * a + bq * bq);
            cs[j] = a / den;
            sn[j] = bq / den;
            H[j * m + j] = den;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            est = fabs(g[j + 1]) / bnorm;
            k = j + 1;
            if (fabs(g[j + 1]) <= rtol * bnorm || hn == 0.0) { conv = 1; break; }
        }
        /* y = H^{-1} g (upper triangular k x k), x += Z y */
        for (int32_t i = k - 1; i >= 0; --i) {
            double s = g[i];
            for (int32_t q = i + 1; q < k; ++q) s -= H[i * m + q] * y[q];
            y[i] = s / H[i * m + i];
        }
        for (int32_t q = 0; q < k; ++q) {
            const double *zq = Z + (size_t)q * nb;
            for (int32_t i = 0; i < nb; ++i) x[i] += y[q] * zq[i];
        }
        if (conv) { rc = 0; break; }
        if (it >= c->o.max_it) { rc = 1; break; }
        ++restarts;
    }
done:
    spmv_rows(&c->A, r0, r1, x, w);
    for (int32_t i = 0; i < nb; ++i) w[i] = bw[i] - w[i];
    st->iters = it;
    st->restarts = restarts;
    st->converged = conv;
    st->est_rel_res = est;
    st->true_rel_res = bnorm > 0.0 ? sqrt(dot(nb, w, w)) / bnorm : 0.0;
    free(bw); free(V); free(Z); free(w); free(H); free(h); free(h2); free(cs); free(sn); free(g); free(y);
    free(full_in); free(full_out);
    return rc;
}

int or_solve(or_ctx *c, const double *rhs, double *x, double rtol, or_stats *st) {
    return fgmres_block(c, 0, c->n, rhs, x, rtol, st);
}

/* FGMRES on one instance of an ensemble set up as a block-diagonal system (cells [cell0,
 * cell0 + ncell)), with the whole system's preconditioner restricted to the block. */
int or_solve_block(or_ctx *c, int32_t cell0, int32_t ncell, const double *rhs, double *x, double rtol,
                   or_stats *st) {
    return fgmres_block(c, cell0, ncell, rhs, x, rtol, st);
}

/* ------------------------------------------------------------------------------------------ */
/* accessors for tests                                                                          */
static amg *pick(or_ctx *c, int which) { return which == 0 ? &c->hp : which == 1 ? &c->hT : &c->hU; }
int or_nlevels(or_ctx *c, int which) { return pick(c, which)->nlev; }
/* info = {n, nnz, nnzP, nc, dense} */
void or_hier_level_info(amg *h, int l, int32_t *info) {
    amg_level *L = &h->L[l];
    info[0] = L->A.n; info[1] = L->A.nnz;
    info[2] = L->P.rp ? L->P.nnz : 0;
    info[3] = (l + 1 < h->nlev) ? h->L[l + 1].A.n : 0;
    info[4] = h->dense;
}
void or_hier_level_get(amg *h, int l, int32_t *rp, int32_t *ci, double *v, double *dinv, int32_t *cf,
                       int32_t *Prp, int32_t *Pci, double *Pv) {
    amg_level *L = &h->L[l];
    memcpy(rp, L->A.rp, sizeof(int32_t) * ((size_t)L->A.n + 1));
    memcpy(ci, L->A.ci, sizeof(int32_t) * (size_t)L->A.nnz);
    memcpy(v, L->A.v, sizeof(double) * (size_t)L->A.nnz);
    memcpy(dinv, L->dinv, sizeof(double) * (size_t)L->A.n);
    if (L->cf && cf) {
        memcpy(cf, L->cf, sizeof(int32_t) * (size_t)L->A.n);
        memcpy(Prp, L->P.rp, sizeof(int32_t) * ((size_t)L->A.n + 1));
        memcpy(Pci, L->P.ci, sizeof(int32_t) * (size_t)L->P.nnz);
        memcpy(Pv, L->P.v, sizeof(double) * (size_t)L->P.nnz);
    }
}
amg *or_hierarchy(or_ctx *c, int which) { return pick(c, which); }
void or_vcycle(or_ctx *c, int which, const double *b, double *x) { vcycle(pick(c, which), 0, b, x); }
void or_stage1(or_ctx *c, const double *v, double *x1) { stage1(c, v, x1); }
void or_ilu_apply(or_ctx *c, const double *r, double *z) { ilu_apply_ordered(c, r, z); }
/* the cell order of the ILU factorisation (new -> original), or identity */
void or_ilu_order(or_ctx *c, int32_t *order) {
    for (int32_t I = 0; I < c->n; ++I) order[I] = c->cperm ? c->cperm[I] : I;
}
void or_spmv(or_ctx *c, const double *x, double *y) { spmv(&c->A, x, y); }
int32_t or_nnz(or_ctx *c) { return c->A.nnz; }
void or_matrix(or_ctx *c, int32_t *rp, int32_t *ci, double *v) {
    memcpy(rp, c->A.rp, sizeof(int32_t) * ((size_t)c->A.n + 1));
    memcpy(ci, c->A.ci, sizeof(int32_t) * (size_t)c->A.nnz);
    memcpy(v, c->A.v, sizeof(double) * (size_t)c->A.nnz);
}
void or_ilu_factors(or_ctx *c, double *v) { memcpy(v, c->ilu.LU.v, sizeof(double) * (size_t)c->ilu.LU.nnz); }
int32_t or_ilu_nnz(or_ctx *c) { return c->ilu.LU.nnz; }
void or_ilu_pattern(or_ctx *c, int32_t *rp, int32_t *ci) {
    memcpy(rp, c->ilu.LU.rp, sizeof(int32_t) * ((size_t)c->ilu.LU.n + 1));
    memcpy(ci, c->ilu.LU.ci, sizeof(int32_t) * (size_t)c->ilu.LU.nnz);
}
/* field: 0 A_pp, 1 A_pT, 2 A_Tp, 3 S~_T (values on their own patterns; S~_T may differ) */
void or_field(or_ctx *c, int f, double *v) {
    const csr *F = f == 0 ? &c->App : f == 1 ? &c->ApT : f == 2 ? &c->ATp : &c->St;
    memcpy(v, F->v, sizeof(double) * (size_t)F->nnz);
}
uint64_t or_splitmix64(uint64_t seed, uint64_t i) { return splitmix64_at(seed, i); }

/* Standalone AMG hierarchy on a scalar CSR matrix (for tests of the AMG pieces in isolation). */
amg *or_amg_create(int32_t n, const int32_t *rp, const int32_t *ci, const double *v, const or_opts *o, int *status) {
    amg *h = (amg *)calloc(1, sizeof(amg));
    csr A;
    A.n = n; A.nnz = rp[n];
    A.rp = (int32_t *)rp; A.ci = (int32_t *)ci; A.v = (double *)v;
    *status = amg_setup(h, &A, o);
    return h;
}
/* Standalone unknown-based AMG on a scalar CSR matrix in unknown-wise order (first np rows: the
 * first unknown). */
amg *or_uamg_create(int32_t n, const int32_t *rp, const int32_t *ci, const double *v, int32_t np, const or_opts *o,
                    int *status) {
    amg *h = (amg *)calloc(1, sizeof(amg));
    csr A;
    A.n = n; A.nnz = rp[n];
    A.rp = (int32_t *)rp; A.ci = (int32_t *)ci; A.v = (double *)v;
    *status = uamg_setup(h, &A, np, o);
    return h;
}
void or_amg_destroy(amg *h) { if (h) { amg_free(h); free(h); } }
void or_amg_vcycle(amg *h, const double *b, double *x) { vcycle(h, 0, b, x); }
int or_amg_nlevels(amg *h) { return h->nlev; }

/* ------------------------------------------------------------------------------------------ */
/* Learned diagonal scaling of the temperature Schur approximation.                             */
/*                                                                                              */
/* The paper approximates S_T = A_TT - A_Tp A_pp^{-1} A_pT by the discrete S_e or, without it,  */
/* by A_TT (Sec. 3.3.1).  The learned form scales the rows of that base approximation B:        */
/* S~_T = diag(s) B, s_i = sinh(y_i), where y_i is the output of a 16-64-64-1 tanh network over */
/* local features of cell i.  The network is trained to regress asinh of the exact ratio        */
/* (S_T)_ii / B_ii.  The paper has no learned part; every choice below (features, target,       */
/* network, optimiser) is this project's.                                                        */

#define OR_NF 16
#define OR_NH 64
/* parameter layout: W1[NH][NF] | b1[NH] | W2[NH][NH] | b2[NH] | w3[NH] | b3 */
#define OR_OFF_W1 0
#define OR_OFF_B1 (OR_OFF_W1 + OR_NH * OR_NF)
#define OR_OFF_W2 (OR_OFF_B1 + OR_NH)
#define OR_OFF_B2 (OR_OFF_W2 + OR_NH * OR_NH)
#define OR_OFF_W3 (OR_OFF_B2 + OR_NH)
#define OR_OFF_B3 (OR_OFF_W3 + OR_NH)
#define OR_NPARAM (OR_OFF_B3 + 1)

int or_mlp_nparam(void) { return OR_NPARAM; }

static double q_div(double x, double y) { return y == 0.0 ? 0.0 : x / y; }
static double sgn(double x) { return x > 0.0 ? 1.0 : x < 0.0 ? -1.0 : 0.0; }

/* value of the cell-pattern field F at (row, col), 0 if the pattern has no such entry */
static double field_at(const csr *F, int32_t row, int32_t col) {
    for (int32_t k = F->rp[row]; k < F->rp[row + 1]; ++k)
        if (F->ci[k] == col) return F->v[k];
    return 0.0;
}

/* entry (r, c) of the diagonal b x b block of cell i of A' (interleaved scalar CSR) */
static double diag_block(const or_ctx *c, int32_t i, int r, int col) {
    const csr *P = &c->App;
    for (int32_t k = P->rp[i]; k < P->rp[i + 1]; ++k)
        if (P->ci[k] == i) return c->A.v[c->A.rp[i * c->b + r] + (k - P->rp[i]) * c->b + col];
    return 0.0;
}

/* The 16 features of every cell (row-major [n][16]); every sum runs over the pattern of row i
 * in ascending position.  B is the base Schur approximation on the cell pattern (S_e when the caller
 * supplies it, else A_TT; values Bv); q(x, y) = x / y (0 when y = 0):
 *   0  q(sum_j A_Tp,ij q(A_pT,ji, A_pp,jj), B_ii)     diagonal of A_Tp D_pp^-1 A_pT, relative
 *   1  q(A_Tp,ii q(A_pT,ii, A_pp,ii), B_ii)           its j = i term
 *   2  q(sum_{j!=i} |A_pp,ij|, |A_pp,ii|)             3  q(sum_{j!=i} |B_ij|, |B_ii|)
 *   4  q(sum_{j!=i} A_pp,ij, |A_pp,ii|)               5  q(sum_{j!=i} B_ij, |B_ii|)
 *   6  q(sum_j |A_Tp,ij q(A_pT,ji, A_pp,jj)|, |B_ii|)
 *   7  q(sum_s a_Ts q(a_sT, a_ss), B_ii)              8  q(sum_s a_ps q(a_sp, a_ss), A_pp,ii)
 *      (a = diagonal block of A', s over the saturation slots)
 *   9  sign(A_pp,ii)                                  10 sign(B_ii)
 *   11 q(A_pT,ii, sqrt|A_pp,ii B_ii|)                  12 q(A_Tp,ii, sqrt|A_pp,ii B_ii|)
 *   13 (entries in row i) / 7
 *   14 q(sum_{j!=i} |A_pT,ij| |A_Tp,ii|, |A_pp,ii B_ii|)
 *   15 q(sum_{j!=i} |A_Tp,ij| |A_pT,ii|, |A_pp,ii B_ii|)
 * and each value v is replaced by asinh(v). */
void or_schur_features(or_ctx *c, const double *Bv, double *feat) {
    int32_t n = c->n, b = c->b;
    csr ATT;   /* B on the cell pattern */
    ATT.n = n; ATT.nnz = c->App.nnz; ATT.rp = c->App.rp; ATT.ci = c->App.ci; ATT.v = (double *)Bv;
    const int32_t *rp = c->App.rp, *ci = c->App.ci;
    for (int32_t i = 0; i < n; ++i) {
        double app = field_at(&c->App, i, i), bii = field_at(&ATT, i, i);
        double apt = field_at(&c->ApT, i, i), atp = field_at(&c->ATp, i, i);
        double s0 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0, s6 = 0, s14 = 0, s15 = 0;
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
            int32_t j = ci[k];
            double t = c->ATp.v[k] * q_div(field_at(&c->ApT, j, i), field_at(&c->App, j, j));
            s0 += t;
            s6 += fabs(t);
            if (j != i) {
                s2 += fabs(c->App.v[k]);
                s3 += fabs(ATT.v[k]);
                s4 += c->App.v[k];
                s5 += ATT.v[k];
                s14 += fabs(c->ApT.v[k]);
                s15 += fabs(c->ATp.v[k]);
            }
        }
        double s7 = 0, s8 = 0;
        for (int s = 0; s < b; ++s) {
            if (s == c->ps || s == c->ts) continue;
            double ass = diag_block(c, i, s, s);
            s7 += diag_block(c, i, c->ts, s) * q_div(diag_block(c, i, s, c->ts), ass);
            s8 += diag_block(c, i, c->ps, s) * q_div(diag_block(c, i, s, c->ps), ass);
        }
        double r = sqrt(fabs(app * bii)), pb = fabs(app * bii);
        double f[OR_NF];
        f[0] = q_div(s0, bii);
        f[1] = q_div(atp * q_div(apt, app), bii);
        f[2] = q_div(s2, fabs(app));
        f[3] = q_div(s3, fabs(bii));
        f[4] = q_div(s4, fabs(app));
        f[5] = q_div(s5, fabs(bii));
        f[6] = q_div(s6, fabs(bii));
        f[7] = q_div(s7, bii);
        f[8] = q_div(s8, app);
        f[9] = sgn(app);
        f[10] = sgn(bii);
        f[11] = q_div(apt, r);
        f[12] = q_div(atp, r);
        f[13] = (double)(rp[i + 1] - rp[i]) / 7.0;
        f[14] = q_div(s14 * fabs(atp), pb);
        f[15] = q_div(s15 * fabs(apt), pb);
        for (int k = 0; k < OR_NF; ++k) feat[(int64_t)i * OR_NF + k] = asinh(f[k]);
    }
}

/* A_TT values on the cell pattern (the base of the learned scaling) */
void or_att(or_ctx *c, double *v) {
    csr ATT;
    extract_field(c, c->App.rp, c->App.ci, c->ts, c->ts, &ATT);
    memcpy(v, ATT.v, sizeof(double) * (size_t)ATT.nnz);
    csr_free(&ATT);
}

/* Forward pass in FP64 for n samples x[n][16]: z1 = W1 x + b1, h1 = tanh z1, z2 = W2 h1 + b2,
 * h2 = tanh z2, y = w3 . h2 + b3. */
static double mlp_forward1(const double *P, const double *x, double *h1, double *h2) {
    for (int j = 0; j < OR_NH; ++j) {
        double z = P[OR_OFF_B1 + j];
        for (int k = 0; k < OR_NF; ++k) z += P[OR_OFF_W1 + j * OR_NF + k] * x[k];
        h1[j] = tanh(z);
    }
    for (int j = 0; j < OR_NH; ++j) {
        double z = P[OR_OFF_B2 + j];
        for (int k = 0; k < OR_NH; ++k) z += P[OR_OFF_W2 + j * OR_NH + k] * h1[k];
        h2[j] = tanh(z);
    }
    double y = P[OR_OFF_B3];
    for (int j = 0; j < OR_NH; ++j) y += P[OR_OFF_W3 + j] * h2[j];
    return y;
}

void or_mlp_forward(const double *P, const double *x, int32_t n, double *y) {
    double h1[OR_NH], h2[OR_NH];
    for (int32_t i = 0; i < n; ++i) y[i] = mlp_forward1(P, x + (int64_t)i * OR_NF, h1, h2);
}

/* Mean squared error L = (1/n) sum_i (y_i - t_i)^2 and its gradient dL/dP by backpropagation
 * (chain rule through the layers above; tanh' = 1 - tanh^2). */
double or_mlp_loss_grad(const double *P, const double *x, const double *t, int32_t n, double *g) {
    double h1[OR_NH], h2[OR_NH], d2[OR_NH], d1[OR_NH];
    memset(g, 0, sizeof(double) * OR_NPARAM);
    double loss = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        const double *xi = x + (int64_t)i * OR_NF;
        double y = mlp_forward1(P, xi, h1, h2);
        double e = y - t[i];
        loss += e * e;
        double dy = 2.0 * e / n;
        g[OR_OFF_B3] += dy;
        for (int j = 0; j < OR_NH; ++j) {
            g[OR_OFF_W3 + j] += dy * h2[j];
            d2[j] = dy * P[OR_OFF_W3 + j] * (1.0 - h2[j] * h2[j]);
        }
        for (int j = 0; j < OR_NH; ++j) {
            g[OR_OFF_B2 + j] += d2[j];
            for (int k = 0; k < OR_NH; ++k) g[OR_OFF_W2 + j * OR_NH + k] += d2[j] * h1[k];
        }
        for (int k = 0; k < OR_NH; ++k) {
            double s = 0.0;
            for (int j = 0; j < OR_NH; ++j) s += P[OR_OFF_W2 + j * OR_NH + k] * d2[j];
            d1[k] = s * (1.0 - h1[k] * h1[k]);
        }
        for (int j = 0; j < OR_NH; ++j) {
            g[OR_OFF_B1 + j] += d1[j];
            for (int k = 0; k < OR_NF; ++k) g[OR_OFF_W1 + j * OR_NF + k] += d1[j] * xi[k];
        }
    }
    return loss / n;
}

/* Adam (Kingma and Ba, 2015): step number t >= 1, moments m, v updated in place. */
void or_adam_step(double *P, double *m, double *v, const double *g, int32_t np, int32_t t, double lr,
                  double beta1, double beta2, double eps) {
    double c1 = 1.0 - pow(beta1, t), c2 = 1.0 - pow(beta2, t);
    for (int32_t p = 0; p < np; ++p) {
        m[p] = beta1 * m[p] + (1.0 - beta1) * g[p];
        v[p] = beta2 * v[p] + (1.0 - beta2) * g[p] * g[p];
        double mh = m[p] / c1, vh = v[p] / c2;
        P[p] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* Inference as the BF16 form computes it: weights (FP32 given) and every layer input rounded to
 * BF16 (features: FP64 -> FP32 -> BF16), biases FP32, each layer's sum accumulated in FP32 from the
 * bias in ascending input order (the BF16 x BF16 products are exact in FP32), tanh in FP32. */
static float f32_tanh(float z) { return tanhf(z); }
void or_mlp_infer_bf16(const float *P, const double *x, int32_t n, float *y) {
    float w1[OR_NH * OR_NF], w2[OR_NH * OR_NH], w3[OR_NH];
    for (int k = 0; k < OR_NH * OR_NF; ++k) w1[k] = (float)round_bf16(P[OR_OFF_W1 + k]);
    for (int k = 0; k < OR_NH * OR_NH; ++k) w2[k] = (float)round_bf16(P[OR_OFF_W2 + k]);
    for (int k = 0; k < OR_NH; ++k) w3[k] = (float)round_bf16(P[OR_OFF_W3 + k]);
    for (int32_t i = 0; i < n; ++i) {
        float xb[OR_NF], h1[OR_NH];
        for (int k = 0; k < OR_NF; ++k) xb[k] = (float)round_bf16(x[(int64_t)i * OR_NF + k]);
        for (int j = 0; j < OR_NH; ++j) {
            float acc = P[OR_OFF_B1 + j];
            for (int k = 0; k < OR_NF; ++k) acc = acc + w1[j * OR_NF + k] * xb[k];
            h1[j] = (float)round_bf16(f32_tanh(acc));
        }
        float out = P[OR_OFF_B3];
        for (int j = 0; j < OR_NH; ++j) {
            float acc = P[OR_OFF_B2 + j];
            for (int k = 0; k < OR_NH; ++k) acc = acc + w2[j * OR_NH + k] * h1[k];
            float h2 = (float)round_bf16(f32_tanh(acc));
            out = out + w3[j] * h2;
        }
        y[i] = out;
    }
}
