// Classical AMG built and applied on the device: strength of connection, PMIS C/F splitting,
// direct interpolation, Galerkin coarse operators A_c = P^T (A P), l1- or omega-Jacobi smoothing
// and a dense inverse on the coarsest level.  Used for A_pp and S~_T in stage 1 of CPTR
// (Sec. 3.3: "Both A_pp^{-1} and S~_T^{-1} are approximated using an AMG V-cycle") and for A_pp
// in CPR (Sec. 3.1).  The set-up arithmetic is ordered so that every value is produced by the
// same sequence of IEEE operations in a fixed order (no fused multiply-add in sums of products):
// the hierarchy is deterministic run to run.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.cuh"

namespace cptr {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ------------------------------------------------------------------------------------------------
// smoother diagonal
__global__ void k_dinv(int32_t n, const int32_t *rp, const int32_t *ci, const double *v, int smoother, double omega,
                       double *dinv) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = 0.0;
    if (smoother == CPTR_SMOOTH_L1) {
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) d = __dadd_rn(d, fabs(v[k]));
        dinv[i] = 1.0 / d;
    } else {
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
            if (ci[k] == i) d = __dadd_rn(d, v[k]);
        dinv[i] = omega / d;
    }
}

// ------------------------------------------------------------------------------------------------
// strength: j != i strong iff -a_ij >= theta * max_{k != i}(-a_ik) > 0.  With an unknown id per
// row (fn, unknown-based AMG of Sec. 3.4), only entries between rows of the same unknown count: the
// classical definitions applied to each diagonal block of a matrix in unknown-wise order.
__device__ __forceinline__ bool same_unknown(const int32_t *fn, int32_t i, int32_t j) { return !fn || fn[i] == fn[j]; }
__device__ __forceinline__ bool row_threshold(const int32_t *rp, const int32_t *ci, const double *v, int32_t i,
                                              double theta, double *thr, const int32_t *fn) {
    double m = 0.0;
    bool have = false;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
        if (ci[k] == i || !same_unknown(fn, i, ci[k])) continue;
        double t = -v[k];
        if (!have || t > m) { m = t; have = true; }
    }
    *thr = theta * m;
    return have && m > 0.0;
}

__global__ void k_strength_count(int32_t n, const int32_t *rp, const int32_t *ci, const double *v, double theta,
                                 int32_t *cnt, const int32_t *fn) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double thr;
    int32_t c = 0;
    if (row_threshold(rp, ci, v, i, theta, &thr, fn))
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) c += (ci[k] != i && same_unknown(fn, i, ci[k]) && -v[k] >= thr);
    cnt[i] = c;
}

__global__ void k_strength_fill(int32_t n, const int32_t *rp, const int32_t *ci, const double *v, double theta,
                                const int32_t *Srp, int32_t *Sci, int32_t *Spos, const int32_t *fn) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double thr;
    int32_t o = Srp[i];
    if (row_threshold(rp, ci, v, i, theta, &thr, fn))
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
            if (ci[k] != i && same_unknown(fn, i, ci[k]) && -v[k] >= thr) { Sci[o] = ci[k]; Spos[o] = k; ++o; }
}

// pattern transpose helpers
// cnt[j] += number of entries of column j among ci[0, nnz) (nnz_dev: the count in device memory
// instead, for a launch sized by an upper bound)
__global__ void k_count_cols(int32_t nnz, const int32_t *ci, int32_t *cnt, const int32_t *nnz_dev = nullptr) {
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < (nnz_dev ? *nnz_dev : nnz)) atomicAdd(cnt + ci[k], 1);
}
__global__ void k_fill_transpose(int32_t n, const int32_t *rp, const int32_t *ci, const double *v, const int32_t *Trp,
                                 int32_t *cursor, int32_t *Tci, double *Tv) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
        int32_t j = ci[k];
        int32_t p = Trp[j] + atomicAdd(cursor + j, 1);
        Tci[p] = i;
        if (Tv) Tv[p] = v[k];
    }
}
// sort every row by column (insertion sort; rows are short), values follow
__global__ void k_sort_rows(int32_t n, const int32_t *rp, int32_t *ci, double *v) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t a = rp[i] + 1; a < rp[i + 1]; ++a) {
        int32_t c = ci[a];
        double x = v ? v[a] : 0.0;
        int32_t b = a - 1;
        while (b >= rp[i] && ci[b] > c) {
            ci[b + 1] = ci[b];
            if (v) v[b + 1] = v[b];
            --b;
        }
        ci[b + 1] = c;
        if (v) v[b + 1] = x;
    }
}

// ------------------------------------------------------------------------------------------------
// PMIS (De Sterck, Yang, Heys 2006), round-synchronous.  key = (|S^T_i| << 32) | hash32, larger
// (key, index) wins; hash32 = top 32 bits of the i-th SplitMix64 output of stream `seed`.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__device__ __forceinline__ bool beats(uint64_t ki, int32_t i, uint64_t kj, int32_t j) {
    return ki > kj || (ki == kj && i > j);
}

// PMIS weights are drawn by the row's index within its unknown (rows [np, n) of the second unknown
// start again at 0), so that each diagonal block is coarsened as it would be on its own
__global__ void k_pmis_init(int32_t n, const int32_t *Srp, const int32_t *Trp, uint64_t seed, uint64_t *key,
                            int32_t *state, const int32_t *fn, int32_t np) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t deg = (uint64_t)(Trp[i + 1] - Trp[i]);
    const int32_t li = (fn && fn[i]) ? i - np : i;
    key[i] = (deg << 32) | (splitmix64_at(seed, (uint64_t)li) >> 32);
    bool isolated = (Srp[i + 1] == Srp[i]) && (Trp[i + 1] == Trp[i]);
    state[i] = isolated ? 2 : 0;
}

__global__ void k_pmis_select(int32_t n, const int32_t *Srp, const int32_t *Sci, const int32_t *Trp,
                              const int32_t *Tci, const uint64_t *key, const int32_t *state, uint8_t *newc) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint8_t ok = 0;
    if (state[i] == 0) {
        ok = 1;
        uint64_t ki = key[i];
        for (int32_t k = Srp[i]; k < Srp[i + 1] && ok; ++k) {
            int32_t j = Sci[k];
            if (state[j] == 0 && !beats(ki, i, key[j], j)) ok = 0;
        }
        for (int32_t k = Trp[i]; k < Trp[i + 1] && ok; ++k) {
            int32_t j = Tci[k];
            if (state[j] == 0 && !beats(ki, i, key[j], j)) ok = 0;
        }
    }
    newc[i] = ok;
}

__global__ void k_pmis_update(int32_t n, const int32_t *Srp, const int32_t *Sci, int32_t *state, const uint8_t *newc,
                              int32_t *undecided) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (newc[i]) { state[i] = 1; return; }
    if (state[i] != 0) return;
    for (int32_t k = Srp[i]; k < Srp[i + 1]; ++k) {
        int32_t j = Sci[k];
        if (newc[j] || state[j] == 1) { state[i] = 2; return; }
    }
    atomicAdd(undecided, 1);
}

__global__ void k_is_c(int32_t n, const int32_t *state, int32_t *isc) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) isc[i] = state[i] == 1;
}

// ------------------------------------------------------------------------------------------------
// direct interpolation (Stueben): F point i with strong C neighbours C_i,
//   w_ij = -alpha a_ij / (a_ii + sum_{k != i, a_ik > 0} a_ik),
//   alpha = sum_{k != i, a_ik < 0} a_ik / sum_{k in C_i} a_ik
__global__ void k_interp_count(int32_t n, const int32_t *Srp, const int32_t *Sci, const int32_t *state, int32_t *cnt) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (state[i] == 1) { cnt[i] = 1; return; }
    int32_t c = 0;
    for (int32_t k = Srp[i]; k < Srp[i + 1]; ++k) c += state[Sci[k]] == 1;
    cnt[i] = c;
}

__global__ void k_interp_fill(int32_t n, const int32_t *rp, const int32_t *ci, const double *v, const int32_t *Srp,
                              const int32_t *Sci, const int32_t *Spos, const int32_t *state, const int32_t *cidx,
                              const int32_t *Prp, int32_t *Pci, double *Pv, const int32_t *fn) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t o = Prp[i];
    if (state[i] == 1) { Pci[o] = cidx[i]; Pv[o] = 1.0; return; }
    if (Prp[i + 1] == o) return;
    double aii = 0.0, sneg = 0.0, spos = 0.0, sc = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
        int32_t j = ci[k];
        if (!same_unknown(fn, i, j)) continue;
        double a = v[k];
        if (j == i) aii = __dadd_rn(aii, a);
        else if (a < 0.0) sneg = __dadd_rn(sneg, a);
        else if (a > 0.0) spos = __dadd_rn(spos, a);
    }
    for (int32_t k = Srp[i]; k < Srp[i + 1]; ++k)
        if (state[Sci[k]] == 1) sc = __dadd_rn(sc, v[Spos[k]]);
    double d = __dadd_rn(aii, spos);
    double alpha = __ddiv_rn(sneg, sc);
    for (int32_t k = Srp[i]; k < Srp[i + 1]; ++k) {
        int32_t j = Sci[k];
        if (state[j] != 1) continue;
        Pci[o] = cidx[j];
        Pv[o] = __ddiv_rn(__dmul_rn(-alpha, v[Spos[k]]), d);
        ++o;
    }
}

// ------------------------------------------------------------------------------------------------
// C = A B by a per-row merge of the B rows selected by A's row.  Every output entry is the sum,
// in ascending position of A's row, of the products a_il * b_lj, accumulated from 0.0 with
// separately rounded multiply and add; output columns ascending.  NUM = false counts entries.
//
// A group of S lanes merges one output row whose A row has m entries, mlo < m <= mhi: lane l of the
// group holds, in slot j, the head of the B row selected by entry j*S + l (K = ceil(m / S) slots).
// Each step finds the smallest head column by a group min-reduction; the products of the
// matching heads are added in ascending entry order (slot by slot, lanes ascending) and lane 0
// of the group writes the entry.  Short rows use groups of 4 or 8 lanes (eight or four rows per
// warp), so that a warp-wide FP64 instruction serves several rows; long rows use the whole warp
// and up to 8 slots.
constexpr int kGemmTinyS = 4, kGemmTinyK = 2;       // m <= 8
constexpr int kGemmSmallS = 8, kGemmSmallK = 4;     // 8 < m <= 32
constexpr int kGemmLargeK = 8;                      // 32 < m <= 256
constexpr int kGemmMaxM = 32 * kGemmLargeK;

template <bool NUM, int S, int KMAX>
__global__ void __launch_bounds__(256) k_spgemm_grp(int32_t n, int32_t mlo, int32_t mhi, const int32_t *__restrict__ Arp,
                                                     const int32_t *__restrict__ Aci, const double *__restrict__ Av,
                                                     const int32_t *__restrict__ Brp, const int32_t *__restrict__ Bci,
                                                     const double *__restrict__ Bv, const int32_t *__restrict__ Crp,
                                                     int32_t *Cci_or_cnt, double *Cv, int32_t *err) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t row = (int32_t)(gt / S);
    const int lane = threadIdx.x & 31, l = lane & (S - 1), gbase = lane & ~(S - 1);
    const unsigned gmask = (S == 32) ? 0xffffffffu : (((1u << S) - 1u) << gbase);
    if (row >= n) return;                      // the whole group
    const int32_t a0 = Arp[row], m = Arp[row + 1] - a0;
    if (m <= mlo) return;
    if (m > mhi) {
        if (mhi >= kGemmMaxM && l == 0) atomicExch(err, 1);
        return;
    }
    const int K = (m + S - 1) / S;             // slots in use, the same for the whole group
    int32_t p[KMAX], e[KMAX];
    double x[KMAX];
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
        p[j] = 0;
        e[j] = 0;
        x[j] = 0.0;
        const int q = j * S + l;
        if (j < K && q < m) {
            const int32_t lj = Aci[a0 + q];
            p[j] = Brp[lj];
            e[j] = Brp[lj + 1];
            x[j] = Av[a0 + q];
        }
    }
    int32_t out = NUM ? Crp[row] : 0;
    int32_t cnt = 0;
    for (;;) {
        int32_t h[KMAX];
        int32_t mn = INT32_MAX;
#pragma unroll
        for (int j = 0; j < KMAX; ++j) {
            h[j] = (j < K && p[j] < e[j]) ? Bci[p[j]] : INT32_MAX;
            mn = min(mn, h[j]);
        }
        if (S == 32) mn = __reduce_min_sync(0xffffffffu, mn);
        else
#pragma unroll
            for (int o = S / 2; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(gmask, mn, o));
        if (mn == INT32_MAX) break;
        if (NUM) {
            double acc = 0.0;
#pragma unroll
            for (int j = 0; j < KMAX; ++j)
                if (j < K) {
                    const bool mt = h[j] == mn;
                    const double q = mt ? __dmul_rn(x[j], Bv[p[j]]) : 0.0;
                    unsigned bm = __ballot_sync(gmask, mt) & gmask;
                    while (bm) {
                        const int src = __ffs(bm) - 1;
                        acc = __dadd_rn(acc, __shfl_sync(gmask, q, src));
                        bm &= bm - 1;
                    }
                }
            if (l == 0) { Cci_or_cnt[out] = mn; Cv[out] = acc; }
            ++out;
        }
#pragma unroll
        for (int j = 0; j < KMAX; ++j)
            if (j < K && h[j] == mn) ++p[j];
        ++cnt;
    }
    if (!NUM && l == 0) Cci_or_cnt[row] = cnt;
}

template <bool NUM>
static void launch_spgemm(Ctx *c, const Csr &A, const Csr &B, const int32_t *Crp, int32_t *Cci_or_cnt, double *Cv) {
    (k_spgemm_grp<NUM, kGemmTinyS, kGemmTinyK><<<nblk((int64_t)A.n * kGemmTinyS, 256), 256, 0, c->stream>>>(
         A.n, 0, kGemmTinyS * kGemmTinyK, A.rp, A.ci, A.v, B.rp, B.ci, B.v, Crp, Cci_or_cnt, Cv, c->flag),
     note_launch());
    (k_spgemm_grp<NUM, kGemmSmallS, kGemmSmallK><<<nblk((int64_t)A.n * kGemmSmallS, 256), 256, 0, c->stream>>>(
         A.n, kGemmTinyS * kGemmTinyK, kGemmSmallS * kGemmSmallK, A.rp, A.ci, A.v, B.rp, B.ci, B.v, Crp, Cci_or_cnt, Cv, c->flag),
     note_launch());
    (k_spgemm_grp<NUM, 32, kGemmLargeK><<<nblk((int64_t)A.n * 32, 256), 256, 0, c->stream>>>(
         A.n, kGemmSmallS * kGemmSmallK, kGemmMaxM, A.rp, A.ci, A.v, B.rp, B.ci, B.v, Crp, Cci_or_cnt, Cv, c->flag),
     note_launch());
}

// ------------------------------------------------------------------------------------------------
// coarsest level: densify and invert by Gauss-Jordan with partial pivoting (one block)
__global__ void k_densify(int32_t n, const int32_t *rp, const int32_t *ci, const double *v, double *D) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) D[(int64_t)i * n + ci[k]] += v[k];
}

__global__ void __launch_bounds__(1024) k_gauss_jordan(int32_t n, double *a, double *inv, int32_t *singular) {
    extern __shared__ double fac[];   // n factors of the pivot column
    __shared__ double red_v[32];
    __shared__ int32_t red_i[32];
    __shared__ int32_t piv_s;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int64_t e = tid; e < (int64_t)n * n; e += nt) inv[e] = ((e / n) == (e % n)) ? 1.0 : 0.0;
    __syncthreads();
    for (int32_t k = 0; k < n; ++k) {
        // pivot: max |a_ik|, i >= k, lowest index on ties
        double best = -1.0;
        int32_t bi = k;
        for (int32_t i = k + tid; i < n; i += nt) {
            double t = fabs(a[(int64_t)i * n + k]);
            if (t > best) { best = t; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            double ob = __shfl_down_sync(0xffffffffu, best, o);
            int32_t oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if ((tid & 31) == 0) { red_v[tid >> 5] = best; red_i[tid >> 5] = bi; }
        __syncthreads();
        if (tid == 0) {
            double bb = -1.0;
            int32_t ii = k;
            for (int w = 0; w < (nt + 31) / 32; ++w)
                if (red_v[w] > bb || (red_v[w] == bb && red_i[w] < ii)) { bb = red_v[w]; ii = red_i[w]; }
            piv_s = (bb > 0.0) ? ii : -1;
            if (bb <= 0.0) *singular = 1;
        }
        __syncthreads();
        int32_t p = piv_s;
        if (p < 0) return;
        if (p != k)
            for (int32_t j = tid; j < n; j += nt) {
                double t = a[(int64_t)k * n + j]; a[(int64_t)k * n + j] = a[(int64_t)p * n + j]; a[(int64_t)p * n + j] = t;
                t = inv[(int64_t)k * n + j]; inv[(int64_t)k * n + j] = inv[(int64_t)p * n + j]; inv[(int64_t)p * n + j] = t;
            }
        __syncthreads();
        double dk = 1.0 / a[(int64_t)k * n + k];
        __syncthreads();
        for (int32_t j = tid; j < n; j += nt) {
            a[(int64_t)k * n + j] *= dk;
            inv[(int64_t)k * n + j] *= dk;
        }
        __syncthreads();
        for (int32_t i = tid; i < n; i += nt) fac[i] = (i == k) ? 0.0 : a[(int64_t)i * n + k];
        __syncthreads();
        for (int64_t e = tid; e < (int64_t)n * n; e += nt) {
            int32_t i = (int32_t)(e / n), j = (int32_t)(e % n);
            double f = fac[i];
            if (f != 0.0) {
                a[e] -= f * a[(int64_t)k * n + j];
                inv[e] -= f * inv[(int64_t)k * n + j];
            }
        }
        __syncthreads();
    }
}

// The same inverse for matrices that fit in shared memory (n <= kGjSmemMax): in-place
// Gauss-Jordan with partial pivoting by rows (the largest |a_ik|, i >= k, lowest index on ties),
// the whole matrix held in shared memory; the row exchanges are undone at the end as column
// exchanges in reverse order, so that the result is A^{-1}.
constexpr int kGjSmemMax = 160;
constexpr int kGjSmemBytes = (kGjSmemMax * kGjSmemMax + kGjSmemMax) * 8 + kGjSmemMax * 4;
constexpr int kGjFacBytes = 200 * 1024;     // the pivot-column buffer of k_gauss_jordan: n <= 25600 (dense_max)
__global__ void __launch_bounds__(1024) k_gauss_jordan_smem(int32_t n, const double *a_in, double *inv,
                                                            int32_t *singular) {
    extern __shared__ double gj[];
    double *a = gj;                       // n x n
    double *fac = gj + (int64_t)n * n;    // n
    int32_t *perm = reinterpret_cast<int32_t *>(fac + n);
    __shared__ double red_v[32];
    __shared__ int32_t red_i[32];
    __shared__ int32_t piv_s;
    __shared__ double dk_s;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int32_t nn = n * n;
    for (int32_t e = tid; e < nn; e += nt) a[e] = a_in[e];
    __syncthreads();
    for (int32_t k = 0; k < n; ++k) {
        double best = -1.0;
        int32_t bi = k;
        for (int32_t i = k + tid; i < n; i += nt) {
            const double t = fabs(a[i * n + k]);
            if (t > best) { best = t; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_down_sync(0xffffffffu, best, o);
            const int32_t oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if ((tid & 31) == 0) { red_v[tid >> 5] = best; red_i[tid >> 5] = bi; }
        __syncthreads();
        if (tid == 0) {
            double bb = -1.0;
            int32_t ii = k;
            for (int w = 0; w < (nt + 31) / 32; ++w)
                if (red_v[w] > bb || (red_v[w] == bb && red_i[w] < ii)) { bb = red_v[w]; ii = red_i[w]; }
            piv_s = (bb > 0.0) ? ii : -1;
            if (bb <= 0.0) *singular = 1;
            perm[k] = ii;
        }
        __syncthreads();
        const int32_t p = piv_s;
        if (p < 0) return;
        if (p != k)
            for (int32_t j = tid; j < n; j += nt) {
                const double t = a[k * n + j];
                a[k * n + j] = a[p * n + j];
                a[p * n + j] = t;
            }
        __syncthreads();
        if (tid == 0) dk_s = 1.0 / a[k * n + k];
        __syncthreads();
        const double dk = dk_s;
        // row k: a_kk <- 1, then the row times 1 / pivot (so a_kk ends as 1 / pivot)
        for (int32_t j = tid; j < n; j += nt) a[k * n + j] = (j == k ? 1.0 : a[k * n + j]) * dk;
        for (int32_t i = tid; i < n; i += nt) fac[i] = (i == k) ? 0.0 : a[i * n + k];
        __syncthreads();
        // other rows: a_ik <- 0, then row_i -= f_i row_k
        for (int32_t e = tid; e < nn; e += nt) {
            const int32_t i = e / n, j = e - i * n;
            const double f = fac[i];
            if (f != 0.0) a[e] = (j == k ? 0.0 : a[e]) - f * a[k * n + j];
        }
        __syncthreads();
    }
    // undo the row exchanges as column exchanges, last first
    for (int32_t k = n - 1; k >= 0; --k) {
        const int32_t p = perm[k];
        if (p != k)
            for (int32_t i = tid; i < n; i += nt) {
                const double t = a[i * n + k];
                a[i * n + k] = a[i * n + p];
                a[i * n + p] = t;
            }
        __syncthreads();
    }
    for (int32_t e = tid; e < nn; e += nt) inv[e] = a[e];
}

// The same inverse for larger matrices, spread over many blocks: the matrix in global memory (row i
// updated by block i mod gridDim.x), block 0 choosing each pivot and staging the pivot row and row k,
// two grid barriers per pivot.  Launched cooperatively (all blocks resident); every barrier wait is
// bounded (flags[3] records a wait that gave up, and every block then returns).
// flags: [0] singular, [1] barrier arrivals, [2] barrier generation, [3] barrier timeout.
constexpr int kGjThreads = 256;
constexpr unsigned long long kGjWaitNs = 500ULL * 1000ULL * 1000ULL;

__device__ __forceinline__ unsigned gj_load_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void gj_store_release(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// all blocks of the grid arrive before any leaves; false (in every thread of the block) if the
// wait gave up or another block's wait had given up
__device__ bool gj_grid_barrier(int32_t *flags) {
    __shared__ int ok_s;
    unsigned *count = reinterpret_cast<unsigned *>(flags + 1), *gen = reinterpret_cast<unsigned *>(flags + 2);
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = gj_load_acquire(gen);
        __threadfence();
        if (atomicAdd(count, 1u) == gridDim.x - 1) {
            atomicExch(count, 0u);
            gj_store_release(gen, g + 1);
        } else {
            unsigned long long t0;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
            while (gj_load_acquire(gen) == g) {
                if (atomicAdd(reinterpret_cast<unsigned *>(flags + 3), 0u)) { ok = 0; break; }
                unsigned long long t;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
                if (t - t0 > kGjWaitNs) {
                    atomicExch(flags + 3, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

__global__ void __launch_bounds__(kGjThreads) k_gauss_jordan_grid(int32_t n, const double *__restrict__ a_in,
                                                                  double *a, double *prow, double *krow,
                                                                  int32_t *perm, int32_t *flags) {
    __shared__ double red_v[kGjThreads / 32];
    __shared__ int32_t red_i[kGjThreads / 32];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int32_t G = gridDim.x, bid = blockIdx.x;
    for (int32_t i = bid; i < n; i += G)
        for (int32_t j = tid; j < n; j += nt) a[(int64_t)i * n + j] = a_in[(int64_t)i * n + j];
    if (!gj_grid_barrier(flags)) return;
    for (int32_t k = 0; k < n; ++k) {
        if (bid == 0) {
            // pivot: max |a_ik|, i >= k, lowest index on ties
            double best = -1.0;
            int32_t bi = k;
            for (int32_t i = k + tid; i < n; i += nt) {
                const double t = fabs(__ldcg(a + (int64_t)i * n + k));
                if (t > best) { best = t; bi = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_down_sync(0xffffffffu, best, o);
                const int32_t oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if ((tid & 31) == 0) { red_v[tid >> 5] = best; red_i[tid >> 5] = bi; }
            __syncthreads();
            if (tid == 0) {
                double bb = -1.0;
                int32_t ii = k;
                for (int w = 0; w < nt / 32; ++w)
                    if (red_v[w] > bb || (red_v[w] == bb && red_i[w] < ii)) { bb = red_v[w]; ii = red_i[w]; }
                red_i[0] = bb > 0.0 ? ii : -1;
                perm[k] = red_i[0];
                if (bb <= 0.0) flags[0] = 1;
            }
            __syncthreads();
            const int32_t p = red_i[0];
            if (p >= 0)
                for (int32_t j = tid; j < n; j += nt) {
                    prow[j] = __ldcg(a + (int64_t)p * n + j);
                    krow[j] = __ldcg(a + (int64_t)k * n + j);
                }
        }
        if (!gj_grid_barrier(flags)) return;
        const int32_t p = __ldcg(perm + k);
        if (p < 0) return;   // singular: every block leaves at the same step
        const double dk = 1.0 / __ldcg(prow + k);
        for (int32_t i = bid; i < n; i += G) {
            double *row = a + (int64_t)i * n;
            if (i == k) {   // the new row k: the pivot row with a_kk <- 1, times 1 / pivot
                for (int32_t j = tid; j < n; j += nt) row[j] = (j == k ? 1.0 : __ldcg(prow + j)) * dk;
                continue;
            }
            const double *src = i == p ? krow : row;   // row p now holds the old row k
            const double f = __ldcg(src + k);
            __syncthreads();   // every thread has f before the thread of column k overwrites it
            if (f != 0.0) {   // a_ik <- 0, then row_i -= f_i (new row k)
                for (int32_t j = tid; j < n; j += nt) {
                    const double nk = (j == k ? 1.0 : __ldcg(prow + j)) * dk;
                    row[j] = (j == k ? 0.0 : __ldcg(src + j)) - f * nk;
                }
            } else if (i == p) {
                for (int32_t j = tid; j < n; j += nt) row[j] = __ldcg(krow + j);
            }
        }
        if (!gj_grid_barrier(flags)) return;
    }
    // undo the row exchanges as column exchanges, last first (one thread per row)
    for (int32_t i = bid + G * tid; i < n; i += G * nt) {
        double *row = a + (int64_t)i * n;
        for (int32_t k = n - 1; k >= 0; --k) {
            const int32_t p = __ldcg(perm + k);
            if (p != k) {
                const double t = row[k];
                row[k] = row[p];
                row[p] = t;
            }
        }
    }
}

void amg_preload() {
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_gauss_jordan_grid);
    cudaFuncGetAttributes(&fa, k_gauss_jordan_smem);
    cudaFuncGetAttributes(&fa, k_gauss_jordan);
}

// ------------------------------------------------------------------------------------------------
// host: one hierarchy
static cptr_status transpose(Ctx *c, const Csr &A, int32_t ncols, Csr &T) {
    T.n = ncols;
    T.nnz = A.nnz;
    int32_t *cnt = nullptr;
    CPTR_TRY(dalloc_t(c, &cnt, (size_t)ncols + 1));
    CPTR_TRY(dalloc_t(c, &T.rp, (size_t)ncols + 1));
    CPTR_TRY(dalloc_t(c, &T.ci, (size_t)A.nnz));
    CPTR_TRY(dalloc_t(c, &T.v, (size_t)A.nnz));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ((size_t)ncols + 1), c->stream));
    (k_count_cols<<<nblk(A.nnz, 256), 256, 0, c->stream>>>(A.nnz, A.ci, cnt), note_launch());
    CPTR_TRY(scan_exclusive(c, cnt, T.rp, ncols, nullptr));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ((size_t)ncols + 1), c->stream));
    (k_fill_transpose<<<nblk(A.n, 256), 256, 0, c->stream>>>(A.n, A.rp, A.ci, A.v, T.rp, cnt, T.ci, T.v), note_launch());
    (k_sort_rows<<<nblk(ncols, 128), 128, 0, c->stream>>>(ncols, T.rp, T.ci, T.v), note_launch());
    CPTR_CUDA_TRY(c, cudaGetLastError());
    dfree(cnt);
    return CPTR_OK;
}

static cptr_status spgemm(Ctx *c, const Csr &A, const Csr &B, int32_t ncb, Csr &C) {
    C.n = A.n;
    CPTR_TRY(dalloc_t(c, &C.rp, (size_t)A.n + 1));
    int32_t *cnt = nullptr;
    CPTR_TRY(dalloc_t(c, &cnt, (size_t)A.n + 1));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(c->flag, 0, sizeof(int32_t), c->stream));
    launch_spgemm<false>(c, A, B, nullptr, cnt, nullptr);
    CPTR_TRY(scan_exclusive(c, cnt, C.rp, A.n, nullptr));
    int32_t rd[2] = {0, 0};   // the entry count and the overflow flag, one synchronisation
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(&rd[0], C.rp + A.n, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(&rd[1], c->flag, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const int32_t total = rd[0], bad = rd[1];
    if (bad) {
        dfree(cnt);
        return c->fail(CPTR_EINVAL, "AMG: a row of the Galerkin product merges more than 256 rows");
    }
    C.nnz = total;
    CPTR_TRY(dalloc_t(c, &C.ci, (size_t)total));
    CPTR_TRY(dalloc_t(c, &C.v, (size_t)total));
    launch_spgemm<true>(c, A, B, C.rp, C.ci, C.v);
    CPTR_CUDA_TRY(c, cudaGetLastError());
    dfree(cnt);
    (void)ncb;
    return CPTR_OK;
}

static cptr_status alloc_level_vectors(Ctx *c, Level &L) {
    size_t n = (size_t)(L.A.n > 0 ? L.A.n : 1);
    CPTR_TRY(dalloc_t(c, &L.dinv, n));
    CPTR_TRY(dalloc_t(c, &L.b, n));
    CPTR_TRY(dalloc_t(c, &L.x, n));
    CPTR_TRY(dalloc_t(c, &L.t, n));
    CPTR_TRY(dalloc_t(c, &L.r, n));
    (k_dinv<<<nblk(L.A.n, 256), 256, 0, c->stream>>>(L.A.n, L.A.rp, L.A.ci, L.A.v, c->o.smoother, c->o.omega, L.dinv), note_launch());
    CPTR_CUDA_TRY(c, cudaGetLastError());
    return CPTR_OK;
}

__global__ void k_coarse_fn(int32_t n, const int32_t *state, const int32_t *cidx, const int32_t *fn, int32_t *fn_c) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && state[i] == 1) fn_c[cidx[i]] = fn[i];
}

// Coarsen level L into P (n x nc) with PMIS + direct interpolation.  *nc_out = 0 if no C points.
// With unknown ids (L.fn), each unknown's diagonal block is coarsened on its own; *fn_c and *np_c
// receive the coarse level's unknown ids and its number of first-unknown rows.
static cptr_status coarsen(Ctx *c, Level &L, int lev, int32_t *nc_out, int32_t **fn_c, int32_t *np_c) {
    const Csr &A = L.A;
    int32_t n = A.n;
    cudaStream_t s = c->stream;
    int32_t *cnt = nullptr, *Srp = nullptr, *Sci = nullptr, *Spos = nullptr, *Trp = nullptr, *Tci = nullptr;
    int32_t *state = nullptr, *cidx = nullptr, *und = nullptr;
    uint64_t *key = nullptr;
    uint8_t *newc = nullptr;
    CPTR_TRY(dalloc_t(c, &cnt, (size_t)n + 1));
    CPTR_TRY(dalloc_t(c, &Srp, (size_t)n + 1));
    (k_strength_count<<<nblk(n, 256), 256, 0, s>>>(n, A.rp, A.ci, A.v, c->o.theta, cnt, L.fn), note_launch());
    // the strength matrix S has at most A's entries: its arrays are allocated by that bound and its
    // entry count stays on the device (Srp[n]), so no host synchronisation is needed here
    CPTR_TRY(scan_exclusive(c, cnt, Srp, n, nullptr));
    const int32_t nnzS_max = A.nnz;
    CPTR_TRY(dalloc_t(c, &Sci, (size_t)nnzS_max));
    CPTR_TRY(dalloc_t(c, &Spos, (size_t)nnzS_max));
    (k_strength_fill<<<nblk(n, 256), 256, 0, s>>>(n, A.rp, A.ci, A.v, c->o.theta, Srp, Sci, Spos, L.fn), note_launch());
    // S^T pattern (neighbour sets; order irrelevant)
    CPTR_TRY(dalloc_t(c, &Trp, (size_t)n + 1));
    CPTR_TRY(dalloc_t(c, &Tci, (size_t)nnzS_max));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ((size_t)n + 1), s));
    (k_count_cols<<<nblk(nnzS_max, 256), 256, 0, s>>>(nnzS_max, Sci, cnt, Srp + n), note_launch());
    CPTR_TRY(scan_exclusive(c, cnt, Trp, n, nullptr));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ((size_t)n + 1), s));
    (k_fill_transpose<<<nblk(n, 256), 256, 0, s>>>(n, Srp, Sci, nullptr, Trp, cnt, Tci, nullptr), note_launch());
    // PMIS rounds
    CPTR_TRY(dalloc_t(c, &key, (size_t)n));
    CPTR_TRY(dalloc_t(c, &state, (size_t)n));
    CPTR_TRY(dalloc_t(c, &newc, (size_t)n));
    CPTR_TRY(dalloc_t(c, &und, 1));
    (k_pmis_init<<<nblk(n, 256), 256, 0, s>>>(n, Srp, Trp, (uint64_t)(int64_t)c->o.seed + (uint64_t)lev, key, state,
                                              L.fn, L.np), note_launch());
    // rounds are launched three at a time between host checks of the undecided count (a round
    // after the last undecided point is decided changes nothing)
    int rounds = 0;
    for (;;) {
        for (int k = 0; k < 3; ++k) {
            (k_pmis_select<<<nblk(n, 256), 256, 0, s>>>(n, Srp, Sci, Trp, Tci, key, state, newc), note_launch());
            CPTR_CUDA_TRY(c, cudaMemsetAsync(und, 0, sizeof(int32_t), s));
            (k_pmis_update<<<nblk(n, 256), 256, 0, s>>>(n, Srp, Sci, state, newc, und), note_launch());
        }
        int32_t h_und = 0;
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(&h_und, und, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CPTR_CUDA_TRY(c, cudaStreamSynchronize(s));
        if (h_und == 0) break;
        if ((rounds += 3) > 100000) return c->fail(CPTR_EINVAL, "AMG: PMIS did not terminate");
    }
    // coarse numbering and the interpolation's row counts (both totals read with one synchronisation;
    // the counts are not needed when no coarse level follows)
    CPTR_TRY(dalloc_t(c, &cidx, (size_t)n + 1));
    (k_is_c<<<nblk(n, 256), 256, 0, s>>>(n, state, cnt), note_launch());
    CPTR_TRY(scan_exclusive(c, cnt, cidx, n, nullptr));
    L.cf = state;
    state = nullptr;
    L.P.n = n;
    CPTR_TRY(dalloc_t(c, &L.P.rp, (size_t)n + 1));
    (k_interp_count<<<nblk(n, 256), 256, 0, s>>>(n, Srp, Sci, L.cf, cnt), note_launch());
    CPTR_TRY(scan_exclusive(c, cnt, L.P.rp, n, nullptr));
    int32_t tot[2] = {0, 0};
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(&tot[0], cidx + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(&tot[1], L.P.rp + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(s));
    const int32_t nc = tot[0];
    *nc_out = nc;
    if (nc > 0 && nc < n) {
        // interpolation
        const int32_t nnzP = tot[1];
        L.P.nnz = nnzP;
        CPTR_TRY(dalloc_t(c, &L.P.ci, (size_t)nnzP));
        CPTR_TRY(dalloc_t(c, &L.P.v, (size_t)nnzP));
        (k_interp_fill<<<nblk(n, 256), 256, 0, s>>>(n, A.rp, A.ci, A.v, Srp, Sci, Spos, L.cf, cidx, L.P.rp, L.P.ci,
                                                   L.P.v, L.fn), note_launch());
        CPTR_CUDA_TRY(c, cudaGetLastError());
        if (L.fn) {   // unknown ids of the coarse points (C points keep their order: pressure first)
            CPTR_TRY(dalloc_t(c, fn_c, (size_t)nc));
            (k_coarse_fn<<<nblk(n, 256), 256, 0, s>>>(n, L.cf, cidx, L.fn, *fn_c), note_launch());
            *np_c = nc;
            if (L.np < n) CPTR_TRY(copy_to_host(c, np_c, cidx + L.np, sizeof(int32_t)));
        }
    }
    dfree(cnt); dfree(Srp); dfree(Sci); dfree(Spos); dfree(Trp); dfree(Tci);
    dfree(key); dfree(newc); dfree(und); dfree(cidx);
    return CPTR_OK;
}

cptr_status amg_setup(Ctx *c, Hier &h, const int32_t *rp, const int32_t *ci, const double *v, int32_t n,
                      const int32_t *fn0, int32_t np0) {
    amg_free(h);
    int32_t nnz = 0;
    CPTR_TRY(copy_to_host(c, &nnz, rp + n, sizeof(int32_t)));
    Csr &A0 = h.L[0].A;
    A0.n = n;
    A0.nnz = nnz;
    CPTR_TRY(dalloc_t(c, &A0.rp, (size_t)n + 1));
    CPTR_TRY(dalloc_t(c, &A0.ci, (size_t)nnz));
    CPTR_TRY(dalloc_t(c, &A0.v, (size_t)nnz));
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(A0.rp, rp, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToDevice, c->stream));
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(A0.ci, ci, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToDevice, c->stream));
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(A0.v, v, sizeof(double) * (size_t)nnz, cudaMemcpyDeviceToDevice, c->stream));
    if (fn0) {   // unknown-based AMG: the unknown of every row, first-unknown rows first
        CPTR_TRY(dalloc_t(c, &h.L[0].fn, (size_t)n));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(h.L[0].fn, fn0, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, c->stream));
        h.L[0].np = np0;
    }
    int maxl = c->o.max_levels < 1 ? 1 : (c->o.max_levels > kMaxLevels ? kMaxLevels : c->o.max_levels);
    int l = 0;
    double nnz_sum = 0.0;
    for (;;) {
        Level &L = h.L[l];
        CPTR_TRY(alloc_level_vectors(c, L));
        nnz_sum += L.A.nnz;
        if (l + 1 >= maxl || L.A.n <= c->o.n_coarse) break;
        int32_t nc = 0, np_c = 0;
        int32_t *fn_c = nullptr;
        double t0 = host_ms();
        CPTR_TRY(coarsen(c, L, l, &nc, &fn_c, &np_c));
        setup_tick(c, SETUP_COARSEN, &t0);
        if (nc == 0 || nc >= L.A.n) {   // no coarsening possible: this level is the coarsest
            csr_free(L.P);
            dfree(L.cf);
            dfree(fn_c);
            L.cf = nullptr;
            break;
        }
        h.L[l + 1].fn = fn_c;
        h.L[l + 1].np = np_c;
        L.nc = nc;
        CPTR_TRY(transpose(c, L.P, nc, L.PT));
        Csr AP;
        CPTR_TRY(spgemm(c, L.A, L.P, nc, AP));
        CPTR_TRY(spgemm(c, L.PT, AP, nc, h.L[l + 1].A));
        csr_free(AP);
        setup_tick(c, SETUP_RAP, &t0);
        ++l;
    }
    h.nlev = l + 1;
    h.op_complexity = nnz_sum / (double)(nnz > 0 ? nnz : 1);
    Level &C = h.L[l];
    int32_t cn = C.A.n;
    h.dense = 0;
    double tc = host_ms();
    if (cn <= c->o.dense_max) {
        // densified on the main stream; inverted on the coarse stream (one block on one SM), which
        // overlaps the rest of the set-up; amg_coarsest_wait joins it before the inverse is used
        if (!c->coarse_stream) CPTR_CUDA_TRY(c, cudaStreamCreateWithFlags(&c->coarse_stream, cudaStreamNonBlocking));
        if (!c->side_fork) CPTR_CUDA_TRY(c, cudaEventCreateWithFlags(&c->side_fork, cudaEventDisableTiming));
        if (!h.gj_done) CPTR_CUDA_TRY(c, cudaEventCreateWithFlags(&h.gj_done, cudaEventDisableTiming));
        if (!h.gj_flag) CPTR_TRY(dalloc_t(c, &h.gj_flag, 4));
        double *D = nullptr;   // the dense matrix, then (multi-block inverse) pivot row, row k, pivots
        CPTR_TRY(dalloc_t(c, &D, (size_t)cn * cn + 3 * (size_t)cn));
        CPTR_TRY(dalloc_t(c, &h.cinv, (size_t)cn * cn));
        CPTR_CUDA_TRY(c, cudaMemsetAsync(D, 0, sizeof(double) * (size_t)cn * cn, c->stream));
        (k_densify<<<nblk(cn, 128), 128, 0, c->stream>>>(cn, C.A.rp, C.A.ci, C.A.v, D), note_launch());
        CPTR_CUDA_TRY(c, cudaMemsetAsync(h.gj_flag, 0, 4 * sizeof(int32_t), c->stream));
        CPTR_CUDA_TRY(c, cudaEventRecord(c->side_fork, c->stream));
        CPTR_CUDA_TRY(c, cudaStreamWaitEvent(c->coarse_stream, c->side_fork, 0));
        cudaStream_t ss = c->coarse_stream;
        // the shared-memory limits are set to the largest size any call uses, so that the two
        // host threads of the set-up, which may run this at the same time, set the same values
        if (cn <= kGjSmemMax) {
            const size_t smem = sizeof(double) * ((size_t)cn * cn + cn) + sizeof(int32_t) * cn;
            CPTR_CUDA_TRY(c, cudaFuncSetAttribute(k_gauss_jordan_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  kGjSmemBytes));
            (k_gauss_jordan_smem<<<1, 1024, smem, ss>>>(cn, D, h.cinv, h.gj_flag), note_launch());
        } else {
            // many blocks, all resident (cooperative launch); one block where that is not available
            int dev = 0, sms = 0, coop = 0, per_sm = 0;
            CPTR_CUDA_TRY(c, cudaGetDevice(&dev));
            CPTR_CUDA_TRY(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            CPTR_CUDA_TRY(c, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
            CPTR_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gauss_jordan_grid, kGjThreads, 0));
            const int G = std::min<int>(sms, cn);
            bool launched = false;
            if (coop && per_sm >= 1 && G >= 2) {
                int32_t n_arg = cn;
                const double *a_in = D;
                double *a_out = h.cinv, *prow = D + (size_t)cn * cn, *krow = prow + cn;
                int32_t *perm = reinterpret_cast<int32_t *>(krow + cn), *flags = h.gj_flag;
                void *args[] = {&n_arg, &a_in, &a_out, &prow, &krow, &perm, &flags};
                launched = cudaLaunchCooperativeKernel((const void *)k_gauss_jordan_grid, dim3(G), dim3(kGjThreads), args,
                                                       0, ss) == cudaSuccess;
                if (launched) note_launch();
                else cudaGetLastError();   // clear the refusal; the one-block kernel follows
            }
            if (!launched) {
                const size_t smem = sizeof(double) * (size_t)(cn > 0 ? cn : 1);
                CPTR_CUDA_TRY(c, cudaFuncSetAttribute(k_gauss_jordan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      kGjFacBytes));
                (k_gauss_jordan<<<1, 1024, smem, ss>>>(cn, D, h.cinv, h.gj_flag), note_launch());
            }
        }
        CPTR_CUDA_TRY(c, cudaGetLastError());
        if (c->pool) CPTR_CUDA_TRY(c, cudaFreeAsync(D, ss));
        else {
            CPTR_CUDA_TRY(c, cudaStreamSynchronize(ss));
            dfree(D);
        }
        CPTR_CUDA_TRY(c, cudaEventRecord(h.gj_done, ss));
        h.gj_pending = true;
        h.dense = 1;
    }
    setup_tick(c, SETUP_COARSEST, &tc);
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return CPTR_OK;
}

// ------------------------------------------------------------------------------------------------
// A_00 = [A_pp A_pT; A_Tp A_TT] in unknown-wise order (Sec. 3.2 eq. A00) from the cell-pattern
// fields: row i < n holds A_pp row i (columns j) then A_pT row i (columns n + j); row n + i holds
// A_Tp row i then A_TT row i.  fn: 0 on the first n rows, 1 on the others.
__global__ void k_build_a00(int32_t n, int32_t nnzb, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const double *__restrict__ App, const double *__restrict__ ApT,
                            const double *__restrict__ ATp, const double *__restrict__ ATT, int32_t *rp0,
                            int32_t *ci0, double *v0, int32_t *fn) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= 2 * n) return;
    const int u = r >= n, i = u ? r - n : r;
    const int32_t a = rp[i], len = rp[i + 1] - a;
    const int32_t o = 2 * (u ? nnzb + a : a);
    rp0[r] = o;
    if (r == 2 * n - 1) rp0[2 * n] = 4 * nnzb;
    fn[r] = u;
    const double *L = u ? ATp : App, *R = u ? ATT : ApT;
    for (int32_t k = 0; k < len; ++k) {
        ci0[o + k] = ci[a + k];
        v0[o + k] = L[a + k];
        ci0[o + len + k] = n + ci[a + k];
        v0[o + len + k] = R[a + k];
    }
}

cptr_status build_a00(Ctx *c, Csr &A, int32_t **fn) {
    const int32_t n = c->n, nnzb = c->nnzb;
    double *ATT = nullptr;
    CPTR_TRY(dalloc_t(c, &ATT, (size_t)nnzb));
    launch_extract(c, c->ts, c->ts, ATT);
    A.n = 2 * n;
    A.nnz = 4 * nnzb;
    CPTR_TRY(dalloc_t(c, &A.rp, 2 * (size_t)n + 1));
    CPTR_TRY(dalloc_t(c, &A.ci, (size_t)A.nnz));
    CPTR_TRY(dalloc_t(c, &A.v, (size_t)A.nnz));
    CPTR_TRY(dalloc_t(c, fn, 2 * (size_t)n));
    (k_build_a00<<<nblk(2 * (int64_t)n, 256), 256, 0, c->stream>>>(n, nnzb, c->rp, c->ci, c->App, c->ApT, c->ATp, ATT,
                                                                   A.rp, A.ci, A.v, *fn), note_launch());
    CPTR_CUDA_TRY(c, cudaGetLastError());
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    dfree(ATT);
    return CPTR_OK;
}

// S~_diag = A_TT - A_Tp diag(A_pp)^{-1} A_pT (Sec. 3.3.1).  B = A_Tp with column k scaled by
// 1 / (A_pp)_kk (the product a * (1 / d), each rounded), C = B A_pT by the Galerkin SpGEMM (every
// entry summed over k ascending from 0, products and sums separately rounded), then A_TT - C on
// the union of the two patterns, columns ascending.
__global__ void k_scale_cols_by_diag_recip(int32_t n, const int32_t *rp, const int32_t *ci, const double *v,
                                           const int32_t *diag, const double *App, double *out) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
        out[k] = __dmul_rn(v[k], __ddiv_rn(1.0, App[diag[ci[k]]]));
}
template <bool FILL>
__global__ void k_union_sub(int32_t n, const int32_t *arp, const int32_t *aci, const double *av, const int32_t *brp,
                            const int32_t *bci, const double *bv, int32_t *cnt_or_rp, int32_t *sci, double *sv) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t a = arp[i], ae = arp[i + 1], b = brp[i], be = brp[i + 1], o = FILL ? cnt_or_rp[i] : 0;
    while (a < ae || b < be) {
        const int32_t ja = a < ae ? aci[a] : INT32_MAX, jb = b < be ? bci[b] : INT32_MAX;
        if (FILL) {
            if (ja == jb) { sci[o] = ja; sv[o] = __dsub_rn(av[a], bv[b]); }
            else if (ja < jb) { sci[o] = ja; sv[o] = av[a]; }
            else { sci[o] = jb; sv[o] = -bv[b]; }
        }
        if (ja <= jb) ++a;
        if (jb <= ja) ++b;
        ++o;
    }
    if (!FILL) cnt_or_rp[i] = o;
}

cptr_status schur_diag(Ctx *c, Csr &S) {
    const int32_t n = c->n, nnzb = c->nnzb;
    cudaStream_t s = c->stream;
    double *ATT = nullptr, *Bv = nullptr;
    CPTR_TRY(dalloc_t(c, &ATT, (size_t)nnzb));
    CPTR_TRY(dalloc_t(c, &Bv, (size_t)nnzb));
    launch_extract(c, c->ts, c->ts, ATT);
    (k_scale_cols_by_diag_recip<<<nblk(n, 256), 256, 0, s>>>(n, c->rp, c->ci, c->ATp, c->diag, c->App, Bv), note_launch());
    Csr B{n, nnzb, c->rp, c->ci, Bv}, PT{n, nnzb, c->rp, c->ci, c->ApT}, C;
    CPTR_TRY(spgemm(c, B, PT, n, C));
    int32_t *cnt = nullptr;
    CPTR_TRY(dalloc_t(c, &cnt, (size_t)n + 1));
    (k_union_sub<false><<<nblk(n, 256), 256, 0, s>>>(n, c->rp, c->ci, ATT, C.rp, C.ci, C.v, cnt, nullptr, nullptr),
     note_launch());
    S.n = n;
    CPTR_TRY(dalloc_t(c, &S.rp, (size_t)n + 1));
    int32_t nnz = 0;
    CPTR_TRY(scan_exclusive(c, cnt, S.rp, n, &nnz));
    S.nnz = nnz;
    CPTR_TRY(dalloc_t(c, &S.ci, (size_t)nnz));
    CPTR_TRY(dalloc_t(c, &S.v, (size_t)nnz));
    (k_union_sub<true><<<nblk(n, 256), 256, 0, s>>>(n, c->rp, c->ci, ATT, C.rp, C.ci, C.v, S.rp, S.ci, S.v),
     note_launch());
    CPTR_CUDA_TRY(c, cudaGetLastError());
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(s));
    csr_free(C);
    dfree(cnt); dfree(ATT); dfree(Bv);
    return CPTR_OK;
}

cptr_status amg_coarsest_wait(Ctx *c, Hier &h) {
    if (!h.gj_pending) return CPTR_OK;
    double t0 = host_ms();
    h.gj_pending = false;
    CPTR_CUDA_TRY(c, cudaStreamWaitEvent(c->stream, h.gj_done, 0));
    int32_t fl[4] = {0, 0, 0, 0};
    CPTR_TRY(copy_to_host(c, fl, h.gj_flag, sizeof(fl)));
    setup_tick(c, SETUP_COARSEST, &t0);
    if (fl[3]) return c->fail(CPTR_ETIMEOUT, "AMG coarsest inverse: a bounded wait gave up");
    if (fl[0]) return c->fail(CPTR_ESINGULAR, "AMG: singular coarsest-level matrix");
    return CPTR_OK;
}

void amg_free(Hier &h) {
    if (h.gj_pending) {   // the side stream may still use the coarsest matrices
        cudaEventSynchronize(h.gj_done);
        h.gj_pending = false;
    }
    for (int l = 0; l < kMaxLevels; ++l) {
        Level &L = h.L[l];
        csr_free(L.A); csr_free(L.P); csr_free(L.PT);
        dfree(L.dinv); dfree(L.cf); dfree(L.b); dfree(L.x); dfree(L.t); dfree(L.r);
        dfree(L.Av_lo); dfree(L.Pv_lo); dfree(L.PTv_lo);
        dfree(L.dinv32); dfree(L.b32); dfree(L.x32); dfree(L.t32); dfree(L.r32);
        dfree(L.fn);
        L = Level{};
    }
    dfree(h.cinv);
    dfree(h.gj_flag);
    h.gj_flag = nullptr;
    dfree(h.ldev64);
    dfree(h.ldev32);
    h.cinv = nullptr;
    h.ldev64 = h.ldev32 = nullptr;
    h.fuse_l0 = -1;
    h.nlev = 0;
    h.dense = 0;
}

// ------------------------------------------------------------------------------------------------
// V(1,1)-cycle kernels, values VT (double, float or bf16), vectors and sums XT (double or float)
__device__ __forceinline__ double vld(const double *p) { return __ldg(p); }
__device__ __forceinline__ float vld(const float *p) { return __ldg(p); }
__device__ __forceinline__ float vld(const bf16 *p) {
    return __bfloat162float(__ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short *>(p))));
}

// pre-smoothing from zero fused with the residual: t = D^{-1} b, r = b - A t
// (TR: t = D^{-1} b was written by the producer of b, so the row reads t instead of D^{-1} and b:
// one multiply fewer per entry, the same values)
template <int G, typename VT, typename XT, bool TR>
__global__ void __launch_bounds__(512) k_vc_down(int32_t n, const int32_t *__restrict__ rp,
                                                  const int32_t *__restrict__ ci, const VT *__restrict__ v,
                                                  const XT *__restrict__ dinv, const XT *__restrict__ b,
                                                  XT *__restrict__ t, XT *__restrict__ r) {
    pdl_wait();
    int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t row = (int32_t)(gid / G);
    int lane = threadIdx.x % G;
    XT acc = 0;
    if (row < n) {
        int32_t k1 = __ldg(rp + row + 1);
        if (G == 1) {
            acc = row_dot_batched<8>(__ldg(rp + row), k1, ci, [&](int32_t k) { return (XT)vld(v + k); },
                                     [&](int32_t j) {
                                         j = (int32_t)chk(j, n, CHK_VC_COL);
                                         return TR ? __ldg(t + j) : __ldg(dinv + j) * __ldg(b + j);
                                     },
                                     acc);
        } else {
            for (int32_t k = __ldg(rp + row) + lane; k < k1; k += G) {
                int32_t j = (int32_t)chk(__ldg(ci + k), n, CHK_VC_COL);
                acc = fma((XT)vld(v + k), TR ? __ldg(t + j) : __ldg(dinv + j) * __ldg(b + j), acc);
            }
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, G);
    if (row < n && lane == 0) {
        XT bi = b[row];
        if (!TR) t[row] = dinv[row] * bi;
        r[row] = bi - acc;
    }
}
// post-smoothing: x = t + D^{-1} (b - A t)
template <int G, typename VT, typename XT>
__global__ void __launch_bounds__(512) k_vc_post(int32_t n, const int32_t *__restrict__ rp,
                                                  const int32_t *__restrict__ ci, const VT *__restrict__ v,
                                                  const XT *__restrict__ dinv, const XT *__restrict__ b,
                                                  const XT *__restrict__ t, XT *__restrict__ x) {
    pdl_wait();
    int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t row = (int32_t)(gid / G);
    int lane = threadIdx.x % G;
    XT acc = 0;
    if (row < n) {
        int32_t k1 = __ldg(rp + row + 1);
        if (G == 1) {
            acc = row_dot_batched<8>(__ldg(rp + row), k1, ci, [&](int32_t k) { return (XT)vld(v + k); },
                                     [&](int32_t j) { return __ldg(t + chk(j, n, CHK_VC_COL)); }, acc);
        } else {
            for (int32_t k = __ldg(rp + row) + lane; k < k1; k += G)
                acc = fma((XT)vld(v + k), __ldg(t + chk(__ldg(ci + k), n, CHK_VC_COL)), acc);
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, G);
    if (row < n && lane == 0) x[row] = t[row] + dinv[row] * (b[row] - acc);
}
// coarsest dense solve x = A_c^{-1} b in FP64 (one warp per row), whatever the vector type
template <typename XT>
__global__ void k_dense_mv(int32_t n, const double *__restrict__ M, const XT *__restrict__ b, XT *__restrict__ x) {
    pdl_wait();
    int32_t row = (int32_t)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    if (row >= n) return;
    double acc = 0.0;
    for (int32_t j = lane; j < n; j += 32) acc = fma(M[(int64_t)row * n + j], (double)b[j], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) x[row] = (XT)acc;
}
template <typename XT>
__global__ void k_diag_scale(int32_t n, const XT *d, const XT *b, XT *x) {
    pdl_wait();
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = d[i] * b[i];
}

template <typename VT, typename XT, bool TR>
static void launch_down_t(cudaStream_t s, const Level &L, const VT *v, const XT *dinv, const XT *b, XT *t, XT *r) {
    const int G = L.sh_A.G ? L.sh_A.G : lanes_for(L.A.n, L.A.nnz), T = L.sh_A.T;
    unsigned grid = nblk((int64_t)L.A.n * G, T);
    const Csr &A = L.A;
    switch (G) {
    case 1: launch_pdl(k_vc_down<1, VT, XT, TR>, grid, T, 0, s, A.n, A.rp, A.ci, v, dinv, b, t, r); break;
    case 2: launch_pdl(k_vc_down<2, VT, XT, TR>, grid, T, 0, s, A.n, A.rp, A.ci, v, dinv, b, t, r); break;
    case 4: launch_pdl(k_vc_down<4, VT, XT, TR>, grid, T, 0, s, A.n, A.rp, A.ci, v, dinv, b, t, r); break;
    case 8: launch_pdl(k_vc_down<8, VT, XT, TR>, grid, T, 0, s, A.n, A.rp, A.ci, v, dinv, b, t, r); break;
    case 16: launch_pdl(k_vc_down<16, VT, XT, TR>, grid, T, 0, s, A.n, A.rp, A.ci, v, dinv, b, t, r); break;
    default: launch_pdl(k_vc_down<32, VT, XT, TR>, grid, T, 0, s, A.n, A.rp, A.ci, v, dinv, b, t, r); break;
    }
}
template <typename VT, typename XT>
static void launch_down(cudaStream_t s, const Level &L, const VT *v, const XT *dinv, const XT *b, XT *t, XT *r,
                        bool t_ready = false) {
    if (t_ready) launch_down_t<VT, XT, true>(s, L, v, dinv, b, t, r);
    else launch_down_t<VT, XT, false>(s, L, v, dinv, b, t, r);
}
template <typename VT, typename XT>
static void launch_post(cudaStream_t s, const Level &L, const VT *v, const XT *dinv, const XT *b, const XT *t, XT *x) {
    const int G = L.sh_A.G ? L.sh_A.G : lanes_for(L.A.n, L.A.nnz), T = L.sh_A.T;
    unsigned grid = nblk((int64_t)L.A.n * G, T);
    const Csr &A = L.A;
    switch (G) {
    case 1: launch_pdl(k_vc_post<1, VT, XT>, grid, T, 0, s, A.n, A.rp, A.ci, v, dinv, b, t, x); break;
    case 2: launch_pdl(k_vc_post<2, VT, XT>, grid, T, 0, s, A.n, A.rp, A.ci, v, dinv, b, t, x); break;
    case 4: launch_pdl(k_vc_post<4, VT, XT>, grid, T, 0, s, A.n, A.rp, A.ci, v, dinv, b, t, x); break;
    case 8: launch_pdl(k_vc_post<8, VT, XT>, grid, T, 0, s, A.n, A.rp, A.ci, v, dinv, b, t, x); break;
    case 16: launch_pdl(k_vc_post<16, VT, XT>, grid, T, 0, s, A.n, A.rp, A.ci, v, dinv, b, t, x); break;
    default: launch_pdl(k_vc_post<32, VT, XT>, grid, T, 0, s, A.n, A.rp, A.ci, v, dinv, b, t, x); break;
    }
}

// per-level views of the arrays used by the FP64 or by the mixed-precision cycle
template <typename XT> struct LevelVecs;
template <> struct LevelVecs<double> {
    static const double *dinv(const Level &L) { return L.dinv; }
    static double *b(const Level &L) { return L.b; }
    static double *x(const Level &L) { return L.x; }
    static double *t(const Level &L) { return L.t; }
    static double *r(const Level &L) { return L.r; }
};
template <> struct LevelVecs<float> {
    static const float *dinv(const Level &L) { return L.dinv32; }
    static float *b(const Level &L) { return L.b32; }
    static float *x(const Level &L) { return L.x32; }
    static float *t(const Level &L) { return L.t32; }
    static float *r(const Level &L) { return L.r32; }
};

// one smoothing/residual/transfer step of level L with its matrix values in storage VT; pf >= 0
// times each kernel as profiling family pf + step (the fine level only)
// (t_ready: this level's t = D^{-1} b was written by the producer of b; the restriction writes the
// coarse level's t = D_c^{-1} b_c for the same reason)
template <typename VT, typename XT>
static void level_down(const Ctx *c, int pf, const Level &L, const Level &C, const VT *Av, const VT *PTv,
                       const XT *b, bool t_ready) {
    using LV = LevelVecs<XT>;
    cudaStream_t s = c->stream;
    int ev = pf < 0 ? -1 : prof_begin(c, pf);
    launch_down<VT, XT>(s, L, Av, LV::dinv(L), b, LV::t(L), LV::r(L), t_ready);    // t = D^-1 b, r = b - A t
    prof_end(c, ev);
    ev = pf < 0 ? -1 : prof_begin(c, pf + 1);
    launch_csr_spmv_t<VT, XT>(s, L.PT.n, L.PT.nnz, L.PT.rp, L.PT.ci, PTv, LV::r(L), LV::b(C), 0, nullptr,
                              L.sh_PT, L.A.n, LV::dinv(C), LV::t(C));                          // b_c = P^T r
    prof_end(c, ev);
}
template <typename VT, typename XT>
static void level_up(const Ctx *c, int pf, const Level &L, const Level &C, const VT *Av, const VT *Pv, const XT *b,
                     XT *x) {
    using LV = LevelVecs<XT>;
    cudaStream_t s = c->stream;
    int ev = pf < 0 ? -1 : prof_begin(c, pf + 2);
    launch_csr_spmv_t<VT, XT>(s, L.P.n, L.P.nnz, L.P.rp, L.P.ci, Pv, LV::x(C), LV::t(L), 2, nullptr,
                              L.sh_P, C.A.n);                                                  // t += P x_c
    prof_end(c, ev);
    ev = pf < 0 ? -1 : prof_begin(c, pf + 3);
    launch_post<VT, XT>(s, L, Av, LV::dinv(L), b, LV::t(L), x);                     // x = t + D^-1 (b - A t)
    prof_end(c, ev);
}

// ------------------------------------------------------------------------------------------------
// Fused coarse levels.  Below a few thousand rows a level's kernels are too small to fill the GPU
// and cost mostly their launch; one block of 1024 threads runs all of them instead, level after
// level, with __syncthreads between the steps: the down path (pre-smoothing from zero fused with
// the residual, restriction) of levels l0 .. lc-1 in one kernel, the coarsest solve as before,
// then the up path (prolongation, post-smoothing) in a second kernel.  Same operations as the
// level kernels (sums in row order).
constexpr int kFuseRows = 300;
constexpr int kFuseThreads = 1024;

template <typename XT>
__device__ __forceinline__ XT ldval(const void *v, int st, int64_t k) {
    if (st == ST_F64) return (XT) static_cast<const double *>(v)[k];
    if (st == ST_F32) return (XT) static_cast<const float *>(v)[k];
    return (XT)__bfloat162float(static_cast<const bf16 *>(v)[k]);
}

template <typename XT>
__global__ void __launch_bounds__(kFuseThreads) k_vc_fused_down(const LevelDev *__restrict__ L, int l0, int lc,
                                                                const XT *b0) {
    pdl_wait();
    for (int l = l0; l < lc; ++l) {
        const LevelDev &A = L[l];
        const XT *b = l == l0 ? b0 : static_cast<const XT *>(A.b);
        const XT *dinv = static_cast<const XT *>(A.dinv);
        XT *t = static_cast<XT *>(A.t), *r = static_cast<XT *>(A.r);
        for (int32_t i = threadIdx.x; i < A.n; i += blockDim.x) {   // t = D^-1 b, r = b - A t
            XT acc = 0;
            for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
                const int32_t j = A.ci[k];
                acc = fma(ldval<XT>(A.v, A.st, k), dinv[j] * b[j], acc);
            }
            const XT bi = b[i];
            t[i] = dinv[i] * bi;
            r[i] = bi - acc;
        }
        __syncthreads();
        const LevelDev &C = L[l + 1];
        XT *bc = static_cast<XT *>(C.b);
        for (int32_t i = threadIdx.x; i < C.n; i += blockDim.x) {   // b_c = P^T r
            XT acc = 0;
            for (int32_t k = A.PTrp[i]; k < A.PTrp[i + 1]; ++k) acc = fma(ldval<XT>(A.PTv, A.st, k), r[A.PTci[k]], acc);
            bc[i] = acc;
        }
        __syncthreads();
    }
}

template <typename XT>
__global__ void __launch_bounds__(kFuseThreads) k_vc_fused_up(const LevelDev *__restrict__ L, int l0, int lc,
                                                              const XT *b0, XT *x0) {
    pdl_wait();
    for (int l = lc - 1; l >= l0; --l) {
        const LevelDev &A = L[l];
        const LevelDev &C = L[l + 1];
        const XT *b = l == l0 ? b0 : static_cast<const XT *>(A.b);
        XT *x = l == l0 ? x0 : static_cast<XT *>(A.x);
        const XT *dinv = static_cast<const XT *>(A.dinv);
        const XT *xc = static_cast<const XT *>(C.x);
        XT *t = static_cast<XT *>(A.t);
        for (int32_t i = threadIdx.x; i < A.n; i += blockDim.x) {   // t += P x_c
            XT acc = 0;
            for (int32_t k = A.Prp[i]; k < A.Prp[i + 1]; ++k) acc = fma(ldval<XT>(A.Pv, A.st, k), xc[A.Pci[k]], acc);
            t[i] += acc;
        }
        __syncthreads();
        for (int32_t i = threadIdx.x; i < A.n; i += blockDim.x) {   // x = t + D^-1 (b - A t)
            XT acc = 0;
            for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k) acc = fma(ldval<XT>(A.v, A.st, k), t[A.ci[k]], acc);
            x[i] = t[i] + dinv[i] * (b[i] - acc);
        }
        __syncthreads();
    }
}

cptr_status amg_fuse_setup(Ctx *c, Hier &h) {
    h.fuse_l0 = -1;
    dfree(h.ldev64);
    dfree(h.ldev32);
    h.ldev64 = h.ldev32 = nullptr;
    const int lc = h.nlev - 1;
    int l0 = lc;
    while (l0 > 0 && h.L[l0 - 1].A.n <= kFuseRows) --l0;
    if (l0 >= lc || lc < 1) return CPTR_OK;   // nothing to fuse
    const bool lo = c->o.precision == CPTR_PREC_MIXED;
    std::vector<LevelDev> d64(h.nlev), d32(h.nlev);
    for (int l = 0; l < h.nlev; ++l) {
        const Level &L = h.L[l];
        LevelDev a{};
        a.n = L.A.n;
        a.rp = L.A.rp; a.ci = L.A.ci;
        a.Prp = L.P.rp; a.Pci = L.P.ci; a.PTrp = L.PT.rp; a.PTci = L.PT.ci;
        LevelDev f = a;
        a.st = ST_F64; a.v = L.A.v; a.Pv = L.P.v; a.PTv = L.PT.v; a.dinv = L.dinv;
        a.b = L.b; a.x = L.x; a.t = L.t; a.r = L.r;
        d64[l] = a;
        if (lo) {
            f.st = L.st; f.v = L.Av_lo; f.Pv = L.Pv_lo; f.PTv = L.PTv_lo; f.dinv = L.dinv32;
            f.b = L.b32; f.x = L.x32; f.t = L.t32; f.r = L.r32;
            d32[l] = f;
        }
    }
    CPTR_TRY(dalloc_t(c, &h.ldev64, (size_t)h.nlev));
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(h.ldev64, d64.data(), sizeof(LevelDev) * h.nlev, cudaMemcpyHostToDevice, c->stream));
    if (lo) {
        CPTR_TRY(dalloc_t(c, &h.ldev32, (size_t)h.nlev));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(h.ldev32, d32.data(), sizeof(LevelDev) * h.nlev, cudaMemcpyHostToDevice, c->stream));
    }
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    h.fuse_l0 = l0;
    return CPTR_OK;
}

template <typename XT>
static void vcycle_level(const Ctx *c, const Hier &h, int l, const XT *b, XT *x, bool t_ready) {
    using LV = LevelVecs<XT>;
    cudaStream_t s = c->stream;
    const Level &L = h.L[l];
    int32_t n = L.A.n;
    const bool lo = sizeof(XT) == 4;
    if (l == h.nlev - 1) {
        if (h.dense) {
            launch_pdl(k_dense_mv<XT>, nblk((int64_t)n * 32, 256), 256, 0, s, n, (const double *)h.cinv, b, x);
        } else {  // two smoothing sweeps from zero
            launch_pdl(k_diag_scale<XT>, nblk(n, 256), 256, 0, s, n, LV::dinv(L), b, LV::t(L));
            if (!lo) launch_post<double, double>(s, L, L.A.v, L.dinv, (const double *)b, L.t, (double *)x);
            else if (L.st == ST_BF16) launch_post<bf16, float>(s, L, (const bf16 *)L.Av_lo, L.dinv32, (const float *)b, L.t32, (float *)x);
            else launch_post<float, float>(s, L, (const float *)L.Av_lo, L.dinv32, (const float *)b, L.t32, (float *)x);
        }
        return;
    }
    if (l == h.fuse_l0 && (lo ? h.ldev32 : h.ldev64)) {   // levels l .. nlev-2 fused
        const LevelDev *ld = lo ? h.ldev32 : h.ldev64;
        const int lc = h.nlev - 1;
        launch_pdl(k_vc_fused_down<XT>, 1, kFuseThreads, 0, s, ld, l, lc, b);
        vcycle_level<XT>(c, h, lc, LV::b(h.L[lc]), LV::x(h.L[lc]), false);
        launch_pdl(k_vc_fused_up<XT>, 1, kFuseThreads, 0, s, ld, l, lc, b, x);
        return;
    }
    const Level &C = h.L[l + 1];
    const int pf = l == 0 ? PF_VC + 4 * (&h == &c->hT) : -1;
    if (!lo) {
        level_down<double, double>(c, pf, L, C, L.A.v, L.PT.v, (const double *)b, t_ready);
        vcycle_level<XT>(c, h, l + 1, LV::b(C), LV::x(C), true);
        level_up<double, double>(c, pf, L, C, L.A.v, L.P.v, (const double *)b, (double *)x);
    } else if (L.st == ST_BF16) {
        level_down<bf16, float>(c, pf, L, C, (const bf16 *)L.Av_lo, (const bf16 *)L.PTv_lo, (const float *)b, t_ready);
        vcycle_level<XT>(c, h, l + 1, LV::b(C), LV::x(C), true);
        level_up<bf16, float>(c, pf, L, C, (const bf16 *)L.Av_lo, (const bf16 *)L.Pv_lo, (const float *)b, (float *)x);
    } else {
        level_down<float, float>(c, pf, L, C, (const float *)L.Av_lo, (const float *)L.PTv_lo, (const float *)b, t_ready);
        vcycle_level<XT>(c, h, l + 1, LV::b(C), LV::x(C), true);
        level_up<float, float>(c, pf, L, C, (const float *)L.Av_lo, (const float *)L.Pv_lo, (const float *)b, (float *)x);
    }
}

void amg_vcycle(const Ctx *c, const Hier &h, const double *b, double *x, bool t_ready) {
    vcycle_level<double>(c, h, 0, b, x, t_ready);
}
void amg_vcycle32(const Ctx *c, const Hier &h, const float *b, float *x, bool t_ready) {
    vcycle_level<float>(c, h, 0, b, x, t_ready);
}

// the mixed-precision copies of a hierarchy: levels 0 and 1 in FP32, levels >= 2 in BF16
// (matrix and transfer values); D^{-1} and work vectors in FP32; the coarsest dense inverse and
// the FP64 arrays are kept
__global__ void k_d2f(const double *src, int64_t n, float *dst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __double2float_rn(src[i]);
}
cptr_status amg_lower_precision(Ctx *c, Hier &h) {
    for (int l = 0; l < h.nlev; ++l) {
        Level &L = h.L[l];
        L.st = l >= 2 ? ST_BF16 : ST_F32;
        CPTR_TRY(to_lower(c, L.A.v, L.A.nnz, L.st, &L.Av_lo));
        if (l + 1 < h.nlev) {
            CPTR_TRY(to_lower(c, L.P.v, L.P.nnz, L.st, &L.Pv_lo));
            CPTR_TRY(to_lower(c, L.PT.v, L.PT.nnz, L.st, &L.PTv_lo));
        }
        size_t n = (size_t)(L.A.n > 0 ? L.A.n : 1);
        for (float **p : {&L.dinv32, &L.b32, &L.x32, &L.t32, &L.r32}) CPTR_TRY(dalloc_t(c, p, n));
        (k_d2f<<<nblk(L.A.n, 256), 256, 0, c->stream>>>(L.dinv, L.A.n, L.dinv32), note_launch());
    }
    CPTR_CUDA_TRY(c, cudaGetLastError());
    return CPTR_OK;
}

// ------------------------------------------------------------------------------------------------
// Autotuner of the V-cycle kernels.  For every non-coarsest level and each of its three kernels
// (smoother + residual on A, restriction P^T, prolongation P), every launch shape G in
// {1, 2, 4, 8, 16, 32} lanes per row x T in {128, 256, 512} threads per block is timed with CUDA
// events over 5 launches after one warm-up launch, on the level's own work vectors and in the
// precision the cycle uses; the fastest is kept.  Shapes are cached by (kernel, rows, entries,
// storage), so repeated set-ups of one workload tune once.  The shapes change only the order of
// the partial sums inside a row (lanes), never which entries are summed.  In FP64 one lane per row
// often wins on GB300: every step of a cross-lane reduction is a warp-wide FP64 addition, and a
// warp-wide FP64 instruction occupies a sub-partition's FP64 pipe for 64 cycles.
namespace {
template <typename F>
Shape pick_shape(Ctx *c, uint64_t key, F &&launch) {
    auto it = c->tune_cache.find(key);
    if (it != c->tune_cache.end()) return it->second;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    Shape best;
    float best_ms = 1e30f;
    for (int G : {1, 2, 4, 8, 16, 32})
        for (int T : {128, 256, 512}) {
            Shape sh;
            sh.G = (int16_t)G;
            sh.T = (int16_t)T;
            launch(sh);
            cudaEventRecord(e0, c->stream);
            for (int r = 0; r < 5; ++r) launch(sh);
            cudaEventRecord(e1, c->stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) { best_ms = ms; best = sh; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->tune_cache[key] = best;
    return best;
}

// operators of about the same size and row length share a tuning (rows in steps of ~9%, average
// row length in steps of ~19%), so that the set-ups of a Newton loop, whose coarse levels change size
// slightly from one Jacobian to the next, reuse the first set-up's shapes
uint64_t tune_key(int kind, const Csr &A, int st) {
    const double n = A.n > 0 ? (double)A.n : 1.0, avg = A.nnz > 0 ? (double)A.nnz / n : 1.0;
    const uint64_t nb = (uint64_t)llround(8.0 * log2(n)), ab = (uint64_t)llround(4.0 * log2(avg) + 64.0);
    return (uint64_t)kind << 60 | (uint64_t)st << 56 | (nb & 0xFFFFull) << 16 | (ab & 0xFFFFull);
}

template <typename VT, typename XT>
void tune_level(Ctx *c, Level &L, Level &C, const VT *Av, const VT *PTv, const VT *Pv) {
    using LV = LevelVecs<XT>;
    cudaStream_t s = c->stream;
    for (XT *p : {LV::b(L), LV::t(L), LV::r(L), LV::x(L)}) cudaMemsetAsync(p, 0, sizeof(XT) * L.A.n, s);
    for (XT *p : {LV::b(C), LV::x(C)}) cudaMemsetAsync(p, 0, sizeof(XT) * C.A.n, s);
    L.sh_A = pick_shape(c, tune_key(1, L.A, L.st), [&](Shape sh) {
        Level tmp = L;
        tmp.sh_A = sh;
        launch_down<VT, XT>(s, tmp, Av, LV::dinv(L), LV::b(L), LV::t(L), LV::r(L));
    });
    L.sh_PT = pick_shape(c, tune_key(2, L.PT, L.st), [&](Shape sh) {
        launch_csr_spmv_t<VT, XT>(s, L.PT.n, L.PT.nnz, L.PT.rp, L.PT.ci, PTv, LV::r(L), LV::b(C), 0, nullptr, sh,
                                  L.A.n);
    });
    L.sh_P = pick_shape(c, tune_key(3, L.P, L.st), [&](Shape sh) {
        launch_csr_spmv_t<VT, XT>(s, L.P.n, L.P.nnz, L.P.rp, L.P.ci, Pv, LV::x(C), LV::t(L), 2, nullptr, sh,
                                  C.A.n);
    });
}
}  // namespace

cptr_status amg_autotune(Ctx *c, Hier &h) {
    const bool lo = c->o.precision == CPTR_PREC_MIXED;
    for (int l = 0; l + 1 < h.nlev; ++l) {
        Level &L = h.L[l], &C = h.L[l + 1];
        if (!lo) tune_level<double, double>(c, L, C, L.A.v, L.PT.v, L.P.v);
        else if (L.st == ST_BF16)
            tune_level<bf16, float>(c, L, C, (const bf16 *)L.Av_lo, (const bf16 *)L.PTv_lo, (const bf16 *)L.Pv_lo);
        else tune_level<float, float>(c, L, C, (const float *)L.Av_lo, (const float *)L.PTv_lo, (const float *)L.Pv_lo);
    }
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    CPTR_CUDA_TRY(c, cudaGetLastError());
    return CPTR_OK;
}

}  // namespace cptr
