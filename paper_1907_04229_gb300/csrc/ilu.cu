// Second stage of CPR/CPTR: block ILU(0) of the decoupled Jacobian A' on its own BSR pattern
// (Sec. 3.1, Sec. 4: "ILU(0) is our default").  Factorisation and triangular solves follow the
// level sets: level(i) = 1 + max level(j) over the rows j that row i depends on, so rows of one
// level are independent.  Pivot blocks are stored inverted in the diagonal slots.  With dense
// b x b blocks this is the same operator as scalar ILU(0) of the interleaved matrix.
#include <cuda_runtime.h>
#include <math.h>

#include <stddef.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <type_traits>
#include <utility>
#include <vector>

#include "common.cuh"
#include "sweep.cuh"

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

// ------------------------------------------------------------------------------------------------
// Triangular solves in one launch per sweep.  Positions t = 0..n-1 enumerate the rows level by
// level; a ticket counter hands out chunks of consecutive positions (32 rows of four lanes each,
// below) to a persistent grid, and a block finishes its chunk before it takes another.  The
// values of an unsolved row hold a sentinel NaN payload; the producer overwrites them with relaxed
// stores and a dependent row polls each value with relaxed loads, so every value doubles as its
// own ready flag.  A row depends only on earlier positions, which belong to chunks held by blocks
// that already run: no deadlock.  Every wait is bounded by kWaitNs of GPU time; a wait that gives
// up sets ks->wait_err and the call reports CPTR_ETIMEOUT.
// Dependency slots are handled kDepGroup at a time (8 for the paired-level tables).
constexpr int kDepGroup = 4;

template <typename T>
__global__ void k_sf_fill(int64_t nvals, T *y, T *z, unsigned *ticket) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const T sent = sentinel_value<T>();
    for (; i < nvals; i += stride) {
        y[i] = sent;
        z[i] = sent;
    }
    if (blockIdx.x == 0 && threadIdx.x < 2) ticket[threadIdx.x] = 0u;
}

// FP32 level-set sweeps, one thread per row (FP32 arithmetic is not limited by the FP64 pipe, and
// this form measured faster than four lanes per row there).  Rows depended on are read in groups
// of up to kDepGroup: all their values are loaded at once
// (relaxed, independent loads), then only the entries still holding the sentinel are polled
// again, with a short sleep between rounds, until the bounded wait gives up.  Every value is
// checked on its own, so producers publish with plain relaxed stores and no fence.

template <int B, typename T>
__device__ __forceinline__ void load_group(const T *base, const int32_t *c, T (*v)[B], KState *ks, int sleep_ns) {
    bool pending = false;
#pragma unroll
    for (int g = 0; g < kDepGroup; ++g)
        if (c[g] >= 0)
#pragma unroll
            for (int q = 0; q < B; ++q) {
                v[g][q] = load_relaxed(base + (int64_t)c[g] * B + q);
                pending |= is_sentinel(v[g][q]);
            }
    if (!pending) return;
    const unsigned long long t0 = gtimer();
    while (pending) {
        __nanosleep(sleep_ns);
        pending = false;
#pragma unroll
        for (int g = 0; g < kDepGroup; ++g)
            if (c[g] >= 0)
#pragma unroll
                for (int q = 0; q < B; ++q)
                    if (is_sentinel(v[g][q])) {
                        v[g][q] = load_relaxed(base + (int64_t)c[g] * B + q);
                        pending |= is_sentinel(v[g][q]);
                    }
        if (pending && gtimer() - t0 > kWaitNs) {
            atomicExch(&ks->wait_err, 1);
#pragma unroll
            for (int g = 0; g < kDepGroup; ++g)
#pragma unroll
                for (int q = 0; q < B; ++q)
                    if (is_sentinel(v[g][q])) v[g][q] = (T)0;
            return;
        }
    }
}

// s -= sum over the dependency slots [o0, o1) of block(slot) * value(dep(slot))
template <int B, typename T>
__device__ __forceinline__ void subtract_deps(T *s, int64_t o0, int64_t o1, int lane, const int32_t *__restrict__ col,
                                              const T *__restrict__ val, const T *vec, KState *ks, int sleep_ns,
                                              int32_t n) {
    for (int64_t sl0 = o0; sl0 < o1; sl0 += kDepGroup) {
        int32_t c[kDepGroup];
#pragma unroll
        for (int g = 0; g < kDepGroup; ++g)
            c[g] = (sl0 + g < o1) ? chk_dep(__ldg(col + (sl0 + g) * 32 + lane), n) : -1;
        T a[kDepGroup][B * B];
#pragma unroll
        for (int g = 0; g < kDepGroup; ++g)
            if (c[g] >= 0)
#pragma unroll
                for (int e = 0; e < B * B; ++e) a[g][e] = __ldg(val + ((sl0 + g) * B * B + e) * 32 + lane);
        T v[kDepGroup][B];
        load_group<B, T>(vec, c, v, ks, sleep_ns);
#pragma unroll
        for (int g = 0; g < kDepGroup; ++g)
            if (c[g] >= 0)
#pragma unroll
                for (int rr = 0; rr < B; ++rr)
#pragma unroll
                    for (int q = 0; q < B; ++q) s[rr] = fma(-a[g][rr * B + q], v[g][q], s[rr]);
    }
}


// y(t) = r(pos[t]) - sum_s L(t, s) y(dep(t, s)).  A persistent grid: each block takes chunks of
// kSfThreads positions in ticket order until none is left.  Factors and y in T, r in RT.
template <int B, typename T, typename RT>
__global__ void __launch_bounds__(kSfThreads) k_ilu_fwd_sf(int32_t n, unsigned *ticket, const int32_t *__restrict__ pos,
                                                          const int64_t *__restrict__ off, const int32_t *__restrict__ col,
                                                          const T *__restrict__ val, const RT *__restrict__ r, T *y,
                                                          KState *ks, const double *never, int sleep_ns) {
    __shared__ unsigned blk;
    const unsigned nchunks = (unsigned)((n + kSfThreads - 1) / kSfThreads);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) blk = atomicAdd(ticket, 1u);
        __syncthreads();
        const unsigned b = blk;
        if (b >= nchunks) return;
        const int32_t t = (int32_t)(b * kSfThreads + threadIdx.x);
        if (t >= n) continue;
        if (never && t == 0) (void)wait_value(never, ks);  // failure injection: a value nobody writes
        const int32_t ch = t >> 5, lane = t & 31;
        const int32_t row = __ldg(pos + t);
        T s[B];
#pragma unroll
        for (int q = 0; q < B; ++q) s[q] = (T)__ldg(r + (int64_t)row * B + q);
        subtract_deps<B, T>(s, __ldg(off + ch), __ldg(off + ch + 1), lane, col, val, y, ks, sleep_ns, n);
#pragma unroll
        for (int q = 0; q < B; ++q) store_relaxed(y + (int64_t)t * B + q, s[q]);
    }
}

// z(t) = D(t)^{-1} (y(bmap[t]) - sum_s U(t, s) z(dep(t, s))); out(pos[t]) = z(t) + x1(pos[t]),
// x1 carrying dp in slot ps and dT in slot ts (vectors of type XT); out is FP64
template <int B, typename T, typename XT>
__global__ void __launch_bounds__(kSfThreads) k_ilu_bwd_sf(int32_t n, unsigned *ticket, const int32_t *__restrict__ pos,
                                                          const int32_t *__restrict__ bmap,
                                                          const int64_t *__restrict__ off, const int32_t *__restrict__ col,
                                                          const T *__restrict__ val, const T *__restrict__ dinv,
                                                          const T *__restrict__ y, T *z, double *__restrict__ out,
                                                          int ps, int ts, const XT *__restrict__ dp,
                                                          const XT *__restrict__ dT, KState *ks, int sleep_ns) {
    __shared__ unsigned blk;
    const unsigned nchunks = (unsigned)((n + kSfThreads - 1) / kSfThreads);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) blk = atomicAdd(ticket + 1, 1u);
        __syncthreads();
        const unsigned b = blk;
        if (b >= nchunks) return;
        const int32_t t = (int32_t)(b * kSfThreads + threadIdx.x);
        if (t >= n) continue;
        const int32_t ch = t >> 5, lane = t & 31;
        const int32_t row = __ldg(pos + t);
        const int32_t tf = __ldg(bmap + t);
        T s[B];
#pragma unroll
        for (int q = 0; q < B; ++q) s[q] = __ldcg(y + (int64_t)tf * B + q);
        // the inverted pivot block does not depend on other rows: load it before the waits
        T dv[B * B];
#pragma unroll
        for (int e = 0; e < B * B; ++e) dv[e] = __ldg(dinv + ((int64_t)ch * B * B + e) * 32 + lane);
        subtract_deps<B, T>(s, __ldg(off + ch), __ldg(off + ch + 1), lane, col, val, z, ks, sleep_ns, n);
        T zi[B];
#pragma unroll
        for (int rr = 0; rr < B; ++rr) {
            T a = 0;
#pragma unroll
            for (int q = 0; q < B; ++q) a = fma(dv[rr * B + q], s[q], a);
            zi[rr] = a;
        }
#pragma unroll
        for (int q = 0; q < B; ++q) store_relaxed(z + (int64_t)t * B + q, zi[q]);
#pragma unroll
        for (int q = 0; q < B; ++q) {
            double add = 0.0;
            if (dp && q == ps) add = (double)dp[row];
            if (dT && q == ts) add = (double)dT[row];
            out[(int64_t)row * B + q] = (double)zi[q] + add;
        }
    }
}


// The same sweeps with a row spread over four lanes, lane q of the group computing component q
// (B <= 4): on GB300 a warp-wide FP64 instruction occupies a sub-partition's FP64 pipe for 64
// cycles, and a level's latency includes the pipe time of its warps' FMAs, so a lane that does one
// component's B FMAs per dependency (instead of a row's B*B) shortens every level.  Each component
// is computed with exactly the operations and order of the per-row kernels above.
constexpr int kSfGroup = 4;                          // lanes per row
constexpr int kSfRowsG = kSfThreads / kSfGroup;      // rows per block chunk

// The rows of a warp advance in lockstep rounds: in each round every unfinished group checks the
// dependency values loaded in the previous round (one L2 round trip), reloads those still holding
// the sentinel, and the groups whose values are all present do their FMAs together, so that a
// warp issues each FP64 instruction once per round rather than once per row that happens to have
// diverged from the others.  No group ever waits for another one (a group that is ready computes
// in the same round), so rows of one warp may depend on each other.  State of a lane: its
// component s of the row, and the dependency slots [sl0, sl0 + DG) in flight (DG = 4 for the
// level-set tables, 8 for the paired-level ones, whose rows have up to 6 dependencies on a 3-D grid,
// and 12 for groups of three levels, up to 10 there).
template <int B, typename T, int DG>
struct SweepLane {
    int64_t sl0, o1;
    int32_t c[DG];
    T a[DG][B];
    T pv[DG];      // component q4 of each dependency's value: each lane of a row polls its own
    T s;
    unsigned long long t0;
    bool waiting;
    int32_t nw;      // rounds waited (the bounded wait reads the clock every eighth round)
    int32_t nrows;   // bound of the dependency positions (index checks)
};

// columns, row q4 of the blocks, and the first loads of component q4 of the values of slots
// sl0, sl0 + H, ..., sl0 + (DG - 1) H (H = 2: a row's slots split between two lane halves)
template <int B, typename T, int DG, int H = 1>
__device__ __forceinline__ void sweep_stage(SweepLane<B, T, DG> &L, int q4, int lane, const int32_t *__restrict__ col,
                                            const T *__restrict__ val, const T *vec) {
#pragma unroll
    for (int g = 0; g < DG; ++g)
        L.c[g] = (L.sl0 + g * H < L.o1) ? chk_dep(__ldg(col + (L.sl0 + g * H) * 32 + lane), L.nrows) : -1;
#pragma unroll
    for (int g = 0; g < DG; ++g)
        if (L.c[g] >= 0) {
#pragma unroll
            for (int q = 0; q < B; ++q) L.a[g][q] = __ldg(val + ((L.sl0 + g * H) * B * B + q4 * B + q) * 32 + lane);
            L.pv[g] = load_relaxed(vec + (int64_t)L.c[g] * B + q4);
        }
}

// One round of a group that is not finished: returns true once all its slots are subtracted.
// *pend tells whether the group still waits on a value after this round.  The lanes of a row
// poll one component each; once all are present, each lane takes the others' by shuffles.
template <int B, typename T, int DG, int H = 1>
__device__ __forceinline__ bool sweep_round(SweepLane<B, T, DG> &L, int q4, int lane, unsigned gmask, int g0,
                                            const int32_t *__restrict__ col, const T *__restrict__ val,
                                            const T *vec, KState *ks, bool *pend) {
    bool p = false;
#pragma unroll
    for (int g = 0; g < DG; ++g)
        if (L.c[g] >= 0) p |= is_sentinel(L.pv[g]);
    p = __any_sync(gmask, p);
    if (p) {
        bool late = false;
        if (!L.waiting) {
            L.t0 = gtimer();
            L.waiting = true;
            L.nw = 0;
        } else if ((++L.nw & 7) == 0) {
            late = gtimer() - L.t0 > kWaitNs;
        }
        // the bounded wait gives up: missing values count as 0 (the lanes of a group count the same
        // rounds, so they all take part in the vote or none)
        if ((L.nw & 7) == 0 && __any_sync(gmask, late)) {
            atomicExch(&ks->wait_err, 1);
#pragma unroll
            for (int g = 0; g < DG; ++g)
                if (is_sentinel(L.pv[g])) L.pv[g] = (T)0;
        } else {
#pragma unroll
            for (int g = 0; g < DG; ++g)
                if (L.c[g] >= 0 && is_sentinel(L.pv[g])) L.pv[g] = load_relaxed(vec + (int64_t)L.c[g] * B + q4);
            *pend = true;
            return false;
        }
    }
    L.waiting = false;
#pragma unroll
    for (int g = 0; g < DG; ++g)
        if (L.c[g] >= 0)
#pragma unroll
            for (int q = 0; q < B; ++q) L.s = fma(-L.a[g][q], __shfl_sync(gmask, L.pv[g], g0 + q), L.s);
    L.sl0 += DG * H;
    if (L.sl0 < L.o1) {
        sweep_stage<B, T, DG, H>(L, q4, lane, col, val, vec);
        *pend = true;
        return false;
    }
    return true;
}

// the part of a paired row's equation that needs no other row's result: s -= sum over the slots
// [coff[ch], coff[ch+1]) of row q4 of block(slot) * src(source(slot)) (none for other rows); with
// H = 2 lane half h takes the slots coff[ch] + h, + h + 2, ...
template <int B, typename T, typename ST, int H = 1>
__device__ __forceinline__ T pair_terms(T s, int q4, int32_t ch, int lane, const int64_t *__restrict__ coff,
                                        const int32_t *__restrict__ ccol, const T *__restrict__ cval,
                                        const ST *__restrict__ src, int32_t n, int h = 0) {
    if (!coff) return s;
    const int64_t c1 = __ldg(coff + ch + 1);
    for (int64_t sl = __ldg(coff + ch) + h; sl < c1; sl += H) {
        int32_t k = __ldg(ccol + sl * 32 + lane);
        if (k < 0) continue;
        k = (int32_t)chk(k, n, CHK_ILU_PAIR);
#pragma unroll
        for (int u = 0; u < B; ++u) s = fma(-__ldg(cval + (sl * B * B + q4 * B + u) * 32 + lane), (T)src[(int64_t)k * B + u], s);
    }
    return s;
}

template <int B, typename T, typename RT, int DG>
__global__ void __launch_bounds__(kSfThreads) k_ilu_fwd_g(int32_t n, unsigned *ticket, const int32_t *__restrict__ pos,
                                                         const int64_t *__restrict__ off, const int32_t *__restrict__ col,
                                                         const T *__restrict__ val, const RT *__restrict__ r, T *y,
                                                         KState *ks, const double *never, int sleep_ns,
                                                         const int64_t *__restrict__ coff,
                                                         const int32_t *__restrict__ ccol, const T *__restrict__ cval) {
    __shared__ unsigned blk;
    const unsigned nchunks = (unsigned)((n + kSfRowsG - 1) / kSfRowsG);
    const int q4 = threadIdx.x & (kSfGroup - 1);
    const int g0 = (threadIdx.x & 31) & ~(kSfGroup - 1);
    const unsigned gmask = ((1u << B) - 1u) << g0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) blk = atomicAdd(ticket, 1u);
        __syncthreads();
        const unsigned b = blk;
        if (b >= nchunks) return;
        const int32_t t = (int32_t)(b * kSfRowsG + threadIdx.x / kSfGroup);
        bool done = t >= n || q4 >= B;
        if (never && t == 0 && q4 == 0) (void)wait_value(never, ks);  // failure injection
        SweepLane<B, T, DG> L;
        const int32_t lane = t & 31;
        if (!done) {
            const int32_t ch = t >> 5;
            L.s = (T)__ldg(r + (int64_t)__ldg(pos + t) * B + q4);
            L.s = pair_terms<B, T, RT>(L.s, q4, ch, lane, coff, ccol, cval, r, n);
            L.nrows = n;
            L.sl0 = __ldg(off + ch);
            L.o1 = __ldg(off + ch + 1);
            L.waiting = false;
            if (L.sl0 < L.o1) sweep_stage<B, T, DG>(L, q4, lane, col, val, y);
            else {
                store_relaxed(y + (int64_t)t * B + q4, L.s);
                done = true;
            }
        }
        while (__any_sync(0xffffffffu, !done)) {
            bool pend = false;
            if (!done && sweep_round<B, T, DG>(L, q4, lane, gmask, g0, col, val, y, ks, &pend)) {
                store_relaxed(y + (int64_t)t * B + q4, L.s);
                done = true;
            }
            if (sleep_ns > 0 && __any_sync(0xffffffffu, pend)) __nanosleep(sleep_ns);
        }
    }
}

// FOLD: the tables' blocks carry the row's inverted pivot (grouped-level backward tables): the row
// starts from D^{-1} y and its sum is the result; otherwise D^{-1} is applied to the sum at the end
template <int B, typename T, typename XT, int DG, bool FOLD = false>
__global__ void __launch_bounds__(kSfThreads) k_ilu_bwd_g(int32_t n, unsigned *ticket, const int32_t *__restrict__ pos,
                                                         const int32_t *__restrict__ bmap,
                                                         const int64_t *__restrict__ off, const int32_t *__restrict__ col,
                                                         const T *__restrict__ val, const T *__restrict__ dinv,
                                                         const T *__restrict__ y, T *z, double *__restrict__ out,
                                                         int ps, int ts, const XT *__restrict__ dp,
                                                         const XT *__restrict__ dT, KState *ks, int sleep_ns,
                                                         const int64_t *__restrict__ coff,
                                                         const int32_t *__restrict__ ccol, const T *__restrict__ cval) {
    __shared__ unsigned blk;
    const unsigned nchunks = (unsigned)((n + kSfRowsG - 1) / kSfRowsG);
    const int q4 = threadIdx.x & (kSfGroup - 1);
    const int g0 = (threadIdx.x & 31) & ~(kSfGroup - 1);
    const unsigned gmask = ((1u << B) - 1u) << g0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) blk = atomicAdd(ticket + 1, 1u);
        __syncthreads();
        const unsigned b = blk;
        if (b >= nchunks) return;
        const int32_t t = (int32_t)(b * kSfRowsG + threadIdx.x / kSfGroup);
        bool done = t >= n || q4 >= B;
        SweepLane<B, T, DG> L;
        const int32_t lane = t & 31;
        T dv[B];
        bool fin = false;
        int32_t row = 0;
        double add = 0.0;
        if (!done) {
            const int32_t ch = t >> 5;
            // inputs that do not depend on other rows are loaded before the rounds
            row = __ldg(pos + t);
            if (dp && q4 == ps) add = (double)dp[row];
            if (dT && q4 == ts) add = (double)dT[row];
            // row q4 of the inverted pivot block does not depend on other rows: load it first
#pragma unroll
            for (int q = 0; q < B; ++q) dv[q] = __ldg(dinv + ((int64_t)ch * B * B + q4 * B + q) * 32 + lane);
            const T *yr = y + (int64_t)__ldg(bmap + t) * B;
            if (FOLD) {
                L.s = (T)0;
#pragma unroll
                for (int q = 0; q < B; ++q) L.s = fma(dv[q], __ldcg(yr + q), L.s);
            } else {
                L.s = __ldcg(yr + q4);
            }
            L.s = pair_terms<B, T, T>(L.s, q4, ch, lane, coff, ccol, cval, y, n);
            L.nrows = n;
            L.sl0 = __ldg(off + ch);
            L.o1 = __ldg(off + ch + 1);
            L.waiting = false;
            if (L.sl0 < L.o1) sweep_stage<B, T, DG>(L, q4, lane, col, val, z);
            else fin = true;
        }
        while (__any_sync(0xffffffffu, !done)) {
            bool pend = false;
            if (!done && (fin || sweep_round<B, T, DG>(L, q4, lane, gmask, g0, col, val, z, ks, &pend))) {
                T a = L.s;
                if (!FOLD) {
                    a = 0;
#pragma unroll
                    for (int q = 0; q < B; ++q) a = fma(dv[q], __shfl_sync(gmask, L.s, g0 + q), a);
                }
                store_relaxed(z + (int64_t)t * B + q4, a);
                out[(int64_t)row * B + q4] = (double)a + add;
                done = true;
            }
            if (sleep_ns > 0 && __any_sync(0xffffffffu, pend)) __nanosleep(sleep_ns);
        }
    }
}

// Whether a row of the warp is ready (every lane of its LPR-lane segment has voted in hv) and not
// yet done (dm: the lanes whose row is done; a row's lanes are done together), from the two
// ballots alone: after the shifts, bit g LPR of x is set iff segment g of hv is full.
template <int LPR>
__device__ __forceinline__ bool ready_rows(unsigned hv, unsigned dm) {
    constexpr unsigned kFirst = LPR == 32 ? 1u : LPR == 16 ? 0x00010001u : LPR == 8 ? 0x01010101u : 0x11111111u;
    unsigned x = hv;
#pragma unroll
    for (int o = 1; o < LPR; o <<= 1) x &= x >> o;
    return (x & ~dm & kFirst) != 0u;
}

// The same sweeps with a row over 4H lanes, H parts of four (H = 2 or 4): part h subtracts the
// row's dependency slots h, h + H, ... (and its share of the right-hand-side terms), lane q of a part
// component q, so that each lane's chain of FP64 instructions is about 1/H as long; when every part
// has subtracted its slots the parts' partial sums are added pairwise (a butterfly: parts 0 + 1, then
// with 2 + 3, the same value in every part) and part 0 finishes the row.  The sums are grouped
// differently from the four-lane kernels above, so values differ from them by rounding only.  Rows
// of a warp advance in the same lockstep rounds.
template <int B, typename T, typename RT, int DG, int H>
__global__ void __launch_bounds__(kSfThreads) k_ilu_fwd_h(int32_t n, unsigned *ticket, const int32_t *__restrict__ pos,
                                                         const int64_t *__restrict__ off, const int32_t *__restrict__ col,
                                                         const T *__restrict__ val, const RT *__restrict__ r, T *y,
                                                         KState *ks, const double *never, int sleep_ns,
                                                         const int64_t *__restrict__ coff,
                                                         const int32_t *__restrict__ ccol, const T *__restrict__ cval) {
    constexpr int LPR = kSfGroup * H, RPB = kSfThreads / LPR;   // lanes per row, rows per block chunk
    constexpr unsigned RMASK = (LPR == 32) ? 0xffffffffu : ((1u << LPR) - 1u);
    __shared__ unsigned blk;
    const unsigned nchunks = (unsigned)((n + RPB - 1) / RPB);
    const int q4 = threadIdx.x & (kSfGroup - 1), h = (threadIdx.x / kSfGroup) & (H - 1);
    const int lw = threadIdx.x & 31, gr = lw & ~(LPR - 1), g0 = gr + kSfGroup * h;
    const unsigned gmask = ((1u << B) - 1u) << g0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) blk = atomicAdd(ticket, 1u);
        __syncthreads();
        const unsigned b = blk;
        if (b >= nchunks) return;
        const int32_t t = (int32_t)(b * RPB + threadIdx.x / LPR);
        const bool idle = t >= n || q4 >= B;   // lanes that compute nothing (they still vote)
        bool done = t >= n, half = idle;       // row finished; this half's slots subtracted
        if (never && t == 0 && q4 == 0 && h == 0) (void)wait_value(never, ks);  // failure injection
        SweepLane<B, T, DG> L;
        L.s = (T)0;
        const int32_t lane = t & 31;
        if (!idle) {
            const int32_t ch = t >> 5;
            if (h == 0) L.s = (T)__ldg(r + (int64_t)__ldg(pos + t) * B + q4);
            L.s = pair_terms<B, T, RT, H>(L.s, q4, ch, lane, coff, ccol, cval, r, n, h);
            L.nrows = n;
            L.sl0 = __ldg(off + ch) + h;
            L.o1 = __ldg(off + ch + 1);
            L.waiting = false;
            if (L.sl0 < L.o1) sweep_stage<B, T, DG, H>(L, q4, lane, col, val, y);
            else half = true;
        }
        // votes per round: the parts' progress and the rows' completion (two ballots), from which
        // every lane also derives whether a row of the warp is ready (ready_rows)
        unsigned dm = __ballot_sync(0xffffffffu, done);
        while (dm != 0xffffffffu) {
            bool pend = false;
            if (!half && sweep_round<B, T, DG, H>(L, q4, lane, gmask, g0, col, val, y, ks, &pend)) half = true;
            // a row is ready once all of its lanes have voted; part 0 stores the parts' sum
            const unsigned hv = __ballot_sync(0xffffffffu, half);
            const bool ready = !done && ((hv >> gr) & RMASK) == RMASK;
            // the parts' sum only in rounds where a row of the warp is ready: an FP64 add issued by
            // every polling warp in every round would hold the FP64 pipe the ready rows need
            if (ready_rows<LPR>(hv, dm)) {
                T sum = L.s;
#pragma unroll
                for (int o = kSfGroup; o < LPR; o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                if (ready && !idle && h == 0) store_relaxed(y + (int64_t)t * B + q4, sum);
            }
            if (ready) done = true;
            if (sleep_ns > 0 && __any_sync(0xffffffffu, pend)) __nanosleep(sleep_ns);
            dm = __ballot_sync(0xffffffffu, done);
        }
    }
}

template <int B, typename T, typename XT, int DG, int H>
__global__ void __launch_bounds__(kSfThreads) k_ilu_bwd_h(int32_t n, unsigned *ticket, const int32_t *__restrict__ pos,
                                                         const int32_t *__restrict__ bmap,
                                                         const int64_t *__restrict__ off, const int32_t *__restrict__ col,
                                                         const T *__restrict__ val, const T *__restrict__ dinv,
                                                         const T *__restrict__ y, T *z, double *__restrict__ out,
                                                         int ps, int ts, const XT *__restrict__ dp,
                                                         const XT *__restrict__ dT, KState *ks, int sleep_ns,
                                                         const int64_t *__restrict__ coff,
                                                         const int32_t *__restrict__ ccol, const T *__restrict__ cval) {
    constexpr int LPR = kSfGroup * H, RPB = kSfThreads / LPR;   // lanes per row, rows per block chunk
    constexpr unsigned RMASK = (LPR == 32) ? 0xffffffffu : ((1u << LPR) - 1u);
    __shared__ unsigned blk;
    const unsigned nchunks = (unsigned)((n + RPB - 1) / RPB);
    const int q4 = threadIdx.x & (kSfGroup - 1), h = (threadIdx.x / kSfGroup) & (H - 1);
    const int lw = threadIdx.x & 31, gr = lw & ~(LPR - 1), g0 = gr + kSfGroup * h;
    const unsigned gmask = ((1u << B) - 1u) << g0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) blk = atomicAdd(ticket + 1, 1u);
        __syncthreads();
        const unsigned b = blk;
        if (b >= nchunks) return;
        const int32_t t = (int32_t)(b * RPB + threadIdx.x / LPR);
        const bool idle = t >= n || q4 >= B;
        bool done = t >= n, half = idle;
        SweepLane<B, T, DG> L;
        L.s = (T)0;
        const int32_t lane = t & 31;
        T dv[B];
#pragma unroll
        for (int q = 0; q < B; ++q) dv[q] = (T)0;
        int32_t row = 0;
        double add = 0.0;
        if (!idle) {
            const int32_t ch = t >> 5;
            row = __ldg(pos + t);
            if (h == 0) {   // the tables carry the row's inverted pivot: start from D^{-1} y
                if (dp && q4 == ps) add = (double)dp[row];
                if (dT && q4 == ts) add = (double)dT[row];
#pragma unroll
                for (int q = 0; q < B; ++q) dv[q] = __ldg(dinv + ((int64_t)ch * B * B + q4 * B + q) * 32 + lane);
                const T *yr = y + (int64_t)__ldg(bmap + t) * B;
#pragma unroll
                for (int q = 0; q < B; ++q) L.s = fma(dv[q], __ldcg(yr + q), L.s);
            }
            L.s = pair_terms<B, T, T, H>(L.s, q4, ch, lane, coff, ccol, cval, y, n, h);
            L.nrows = n;
            L.sl0 = __ldg(off + ch) + h;
            L.o1 = __ldg(off + ch + 1);
            L.waiting = false;
            if (L.sl0 < L.o1) sweep_stage<B, T, DG, H>(L, q4, lane, col, val, z);
            else half = true;
        }
        unsigned dm = __ballot_sync(0xffffffffu, done);
        while (dm != 0xffffffffu) {
            bool pend = false;
            if (!half && sweep_round<B, T, DG, H>(L, q4, lane, gmask, g0, col, val, z, ks, &pend)) half = true;
            const unsigned hv = __ballot_sync(0xffffffffu, half);
            const bool ready = !done && ((hv >> gr) & RMASK) == RMASK;
            if (ready_rows<LPR>(hv, dm)) {   // (the parts' sum only when a row is ready)
                T sum = L.s;
#pragma unroll
                for (int o = kSfGroup; o < LPR; o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                if (ready && !idle && h == 0) {
                    store_relaxed(z + (int64_t)t * B + q4, sum);
                    out[(int64_t)row * B + q4] = (double)sum + add;
                }
            }
            if (ready) done = true;
            if (sleep_ns > 0 && __any_sync(0xffffffffu, pend)) __nanosleep(sleep_ns);
            dm = __ballot_sync(0xffffffffu, done);
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Chunked wavefront sweeps.  The rows of the factor order are cut into chunks of K consecutive
// rows (K = the matrix's bandwidth, so that every dependency outside a chunk lies in an earlier
// chunk of the sweep).  One block solves one chunk: it walks the chunk's own level sets (levels
// counted over dependencies inside the chunk) with a __syncthreads between levels, keeping the
// values of the last W levels in a shared-memory ring; dependencies on other chunks (and on
// in-chunk rows more than W-1 levels back) are read from the global vector, whose unsolved
// entries hold the sentinel, with bounded polls.  Chunks are handed out in sweep order by a
// ticket, so a chunk only waits on chunks held by running blocks (no deadlock), and consecutive
// chunks pipeline: on a natural-order grid a chunk is a plane and trails the previous plane by a
// few levels.  The factor blocks of the next level are staged in shared memory by cp.async while
// the current level computes, and the next level's outside dependencies are loaded early.
// Each value is computed exactly as in the level-set sweeps above (same operations, same order).
constexpr int kCwMaxD = 4;
constexpr int kCwMaxThreads = 256;   // the widest level a chunk may have
constexpr int kCwLead = 4;           // levels a chunk runs ahead of the next before that one starts
constexpr int32_t kCwNone = INT32_MIN;

__device__ __forceinline__ void cp_async_elem(double *dst, const double *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_elem(float *dst, const float *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
template <int NS>
__device__ __forceinline__ void cp_async_wait_ns() {   // all but the NS - 1 most recent groups
    asm volatile("cp.async.wait_group %0;" ::"n"(NS - 1) : "memory");
}

// Software pipeline of one chunk, all through shared memory (no register copies of loads in
// flight).  Group g_l, committed at iteration l, copies by cp.async: the row index and dependency
// codes of level l + 2S (position-indexed), the factor blocks of level l + S (position-indexed),
// and the right-hand side and outside-dependency values of level l + S (addresses from the row
// and codes of level l + S, which arrived with g_{l-S}).  Iteration l first waits for g_{l-S}
// (at most S - 1 newer groups pending), so every copy has S levels of work to arrive.  Values of
// outside dependencies that were still unwritten when copied hold the sentinel and are polled
// from global memory when used.
// 16 bytes through L2 only (values another block may have just written must not come from L1)
__device__ __forceinline__ void cp_async_cg16(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_i32(int32_t *dst, const int32_t *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
template <int S>
__device__ __forceinline__ void cp_async_wait_slack() {   // all but the S - 1 most recent groups
    asm volatile("cp.async.wait_group %0;" ::"n"(S - 1) : "memory");
}

// the value of dependency d: from the ring, or the staged copy (polled until written)
template <int B, typename T>
__device__ __forceinline__ void cw_dep(int32_t cd, const T *staged, const T *ring, const T *vec, T *v, KState *ks,
                                       int sleep_ns) {
    if (cd >= 0) {
#pragma unroll
        for (int q = 0; q < B; ++q) v[q] = ring[(int64_t)cd * B + q];
        return;
    }
    const int64_t j = -(int64_t)cd - 1;
    bool pending = false;
#pragma unroll
    for (int q = 0; q < B; ++q) {
        v[q] = staged[q];
        pending |= is_sentinel(v[q]);
    }
    if (!pending) return;
    const unsigned long long t0 = gtimer();
    for (;;) {
        pending = false;
#pragma unroll
        for (int q = 0; q < B; ++q)
            if (is_sentinel(v[q])) {
                v[q] = load_relaxed(vec + j * B + q);
                pending |= is_sentinel(v[q]);
            }
        if (!pending) return;
        if (gtimer() - t0 > kWaitNs) {
            atomicExch(&ks->wait_err, 1);
#pragma unroll
            for (int q = 0; q < B; ++q)
                if (is_sentinel(v[q])) v[q] = (T)0;
            return;
        }
        __nanosleep(sleep_ns);
    }
}

// shared-memory layout of the pipeline (per block), in this order: ring [W][maxw][B] (T);
// blocks [S+1][threads][SW] (T); values [S+1][threads][D][B] (T); rhs [S+1][threads][B] (ST);
// rows [2S+1][threads] and codes [2S+1][D][threads] (int32); level pointers [maxlev+1] (int32)
// every region starts on a 16-byte boundary (the host computes the same sizes: cw_smem_bytes)
__host__ __device__ inline size_t cw_align16(size_t x) { return (x + 15) & ~(size_t)15; }
template <int B, typename T, typename ST>
struct CwSmem {
    T *ring, *blk, *gv;
    ST *rhs;
    int32_t *row, *cd, *lv;
    __device__ CwSmem(unsigned char *base, int W, int maxw, int S, int nthr, int SW, int D) {
        size_t o = 0;
        ring = reinterpret_cast<T *>(base + o);
        o += cw_align16(sizeof(T) * (size_t)W * maxw * B);
        blk = reinterpret_cast<T *>(base + o);
        o += cw_align16(sizeof(T) * (size_t)(S + 1) * nthr * SW);
        gv = reinterpret_cast<T *>(base + o);
        o += cw_align16((size_t)32 * (S + 1) * nthr * D);
        rhs = reinterpret_cast<ST *>(base + o);
        o += cw_align16(sizeof(ST) * (size_t)(S + 1) * nthr * B);
        row = reinterpret_cast<int32_t *>(base + o);
        o += cw_align16(4 * (size_t)(2 * S + 1) * nthr);
        cd = reinterpret_cast<int32_t *>(base + o);
        o += cw_align16(4 * (size_t)(2 * S + 1) * D * nthr);
        lv = reinterpret_cast<int32_t *>(base + o);
    }
};

// One kernel for both sweeps.  Forward (FWD): y(row) = r(row) - sum_d L(row, d) y(dep d).
// Backward: z(row) = D(row)^{-1} (y(row) - sum_d U(row, d) z(dep d)), out(row) = z(row) + x1(row).
// src: r (forward, type ST) or y (backward); vec: the vector being solved (y or z).
template <int B, typename T, typename ST, typename XT, bool FWD, int S>
__global__ void __launch_bounds__(256) k_ilu_cw(int32_t nchunks, int32_t n, int D, int W, int maxw, int maxlev,
                                                unsigned *ticket, const int32_t *__restrict__ clev,
                                                const int32_t *__restrict__ lptr, const int32_t *__restrict__ prow,
                                                const int32_t *__restrict__ code, const T *__restrict__ val,
                                                const ST *__restrict__ src, T *vec, double *__restrict__ out, int ps,
                                                int ts, const XT *__restrict__ dp, const XT *__restrict__ dT,
                                                KState *ks, const double *never, int sleep_ns, int32_t *started,
                                                int lead) {
    constexpr int BB = B * B, NA = 2 * S + 1, NB = S + 1;
    const int SW = FWD ? D * BB : D * BB + BB;
    const int nthr = blockDim.x, tid = threadIdx.x;
    extern __shared__ __align__(16) unsigned char cw_smem[];
    CwSmem<B, T, ST> sm(cw_smem, W, maxw, S, nthr, SW, D);
    __shared__ unsigned chunk_s;
    for (;;) {
        __syncthreads();
        if (tid == 0) chunk_s = atomicAdd(ticket + (FWD ? 0 : 1), 1u);
        __syncthreads();
        const unsigned ch = chunk_s;
        if (ch >= (unsigned)nchunks) return;
        const int L0 = __ldg(clev + ch), nl = __ldg(clev + ch + 1) - L0;
        for (int q = tid; q <= nl; q += nthr) sm.lv[q] = __ldg(lptr + L0 + q);
        if (FWD && never && ch == 0 && tid == 0) (void)wait_value(never, ks);   // failure injection
        if (ch > 0 && tid == 0) {   // the previous chunk has finished its first `lead` levels
            const unsigned long long t0 = gtimer();
            for (;;) {
                int32_t f;
                asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(f) : "l"(started + ch - 1) : "memory");
                if (f) break;
                if (gtimer() - t0 > kWaitNs) { atomicExch(&ks->wait_err, 1); break; }
                __nanosleep(sleep_ns);
            }
        }
        __syncthreads();
        const int lead_level = min(lead, nl) - 1;
        // copies of level m into its slots: A part (row, codes), blocks, B part (rhs, values)
        auto copyA = [&](int m) {
            const int32_t p = sm.lv[m] + tid;
            if (p >= sm.lv[m + 1]) return;
            const int sa = m % NA;
            cp_async_i32(sm.row + sa * nthr + tid, prow + p);
            for (int d = 0; d < D; ++d) cp_async_i32(sm.cd + ((int64_t)sa * D + d) * nthr + tid, code + (int64_t)d * n + p);
        };
        auto copyB = [&](int m) {   // needs the A part of level m in shared memory
            const int32_t p = sm.lv[m] + tid;
            if (p >= sm.lv[m + 1]) return;
            const int sa = m % NA, sb = m % NB;
            const int32_t row = sm.row[sa * nthr + tid];
            for (int e = 0; e < SW; ++e)
                cp_async_elem(sm.blk + ((int64_t)sb * nthr + tid) * SW + e, val + (int64_t)e * n + p);
            for (int q = 0; q < B; ++q)
                cp_async_elem(sm.rhs + ((int64_t)sb * nthr + tid) * B + q, src + (int64_t)row * B + q);
            for (int d = 0; d < D; ++d) {
                const int32_t cd = sm.cd[((int64_t)sa * D + d) * nthr + tid];
                if (cd != kCwNone && cd < 0) {
                    const int64_t j = -(int64_t)cd - 1;
                    const uintptr_t at = reinterpret_cast<uintptr_t>(vec + j * B) & ~(uintptr_t)15;
                    unsigned char *dst = reinterpret_cast<unsigned char *>(sm.gv) + (((int64_t)sb * nthr + tid) * D + d) * 32;
                    cp_async_cg16(dst, reinterpret_cast<const void *>(at));
                    cp_async_cg16(dst + 16, reinterpret_cast<const void *>(at + 16));
                }
            }
        };
        // prologue: A of levels 0 .. 2S-1 (S groups of two levels), then B of levels 0 .. S-1
        for (int k = 0; k < S; ++k) {
            if (2 * k < nl) copyA(2 * k);
            if (2 * k + 1 < nl) copyA(2 * k + 1);
            cp_async_commit();
        }
        cp_async_wait_0();
        for (int k = 0; k < S; ++k) {
            if (k < nl) copyB(k);
            cp_async_commit();
        }
        for (int l = 0; l < nl; ++l) {
            cp_async_wait_slack<S>();            // g_{l-S} (or the prologue group of level l) is complete
            if (l + 2 * S < nl) copyA(l + 2 * S);
            if (l + S < nl) copyB(l + S);        // its A part arrived S iterations ago
            cp_async_commit();
            const int32_t p = sm.lv[l] + tid;
            if (p < sm.lv[l + 1]) {
                const int sa = l % NA, sb = l % NB;
                const int32_t row = sm.row[sa * nthr + tid];
                const T *a = sm.blk + ((int64_t)sb * nthr + tid) * SW;
                const ST *rh = sm.rhs + ((int64_t)sb * nthr + tid) * B;
                T s[B];
#pragma unroll
                for (int q = 0; q < B; ++q) s[q] = (T)rh[q];
                for (int d = 0; d < D; ++d) {
                    const int32_t cd = sm.cd[((int64_t)sa * D + d) * nthr + tid];
                    if (cd == kCwNone) continue;
                    T v[B];
                    const T *win = reinterpret_cast<const T *>(reinterpret_cast<const unsigned char *>(sm.gv) +
                                                               (((int64_t)sb * nthr + tid) * D + d) * 32);
                    const int64_t jj = cd < 0 && cd != kCwNone ? -(int64_t)cd - 1 : 0;
                    const int skew = (int)((reinterpret_cast<uintptr_t>(vec + jj * B) & 15) / sizeof(T));
                    cw_dep<B, T>(cd, win + skew, sm.ring, vec, v, ks, sleep_ns);
                    const T *m = a + d * BB;
#pragma unroll
                    for (int rr = 0; rr < B; ++rr)
#pragma unroll
                        for (int q = 0; q < B; ++q) s[rr] = fma(-m[rr * B + q], v[q], s[rr]);
                }
                T res[B];
                if (FWD) {
#pragma unroll
                    for (int q = 0; q < B; ++q) res[q] = s[q];
                } else {
                    const T *dinv = a + D * BB;
#pragma unroll
                    for (int rr = 0; rr < B; ++rr) {
                        T acc = 0;
#pragma unroll
                        for (int q = 0; q < B; ++q) acc = fma(dinv[rr * B + q], s[q], acc);
                        res[rr] = acc;
                    }
                }
                T *slot = sm.ring + ((int64_t)(l % W) * maxw + tid) * B;
#pragma unroll
                for (int q = 0; q < B; ++q) {
                    slot[q] = res[q];
                    store_relaxed(vec + (int64_t)row * B + q, res[q]);
                    if (!FWD) {
                        double add = 0.0;
                        if (dp && q == ps) add = (double)dp[row];
                        if (dT && q == ts) add = (double)dT[row];
                        out[(int64_t)row * B + q] = (double)res[q] + add;
                    }
                }
            }
            __syncthreads();
            if (l == lead_level && tid == 0)
                asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(started + ch), "r"(1) : "memory");
        }
        cp_async_wait_0();
    }
}

// gather factor blocks into the chunked tables: value e of slot d of position p (plane
// (d * BB + e), entry p) comes from block kidx[d * n + p] (zero where there is none)
template <typename T>
__global__ void k_cw_pack(int32_t n, int nslots, int BB, const int32_t *kidx, const double *LU, T *val) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= (int64_t)nslots * n) return;
    const int d = (int)(u / n);
    const int32_t p = (int32_t)(u % n);
    const int32_t k = kidx[u];
    for (int e = 0; e < BB; ++e) val[((int64_t)d * BB + e) * n + p] = k >= 0 ? (T)LU[(int64_t)k * BB + e] : (T)0;
}

// pack factor blocks into the SELL-32 layout: slot u (slot * 32 + lane) takes block kidx[u]
template <typename T>
__global__ void k_sf_pack(int64_t nslots32, int BB, const int32_t *kidx, const double *LU, T *val) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nslots32) return;
    int64_t sl = u >> 5;
    int lane = (int)(u & 31);
    int32_t k = kidx[u];
    for (int e = 0; e < BB; ++e) val[(sl * BB + e) * 32 + lane] = (T)(k >= 0 ? LU[(int64_t)k * BB + e] : 0.0);
}

// ------------------------------------------------------------------------------------------------
// Set-up of the sweeps on the device.  Level sets in one launch: every row's level is 1 + the
// largest level among the rows it depends on (lower columns forward, upper columns backward), 0
// without dependencies.  Rows are taken by a ticket counter in a topological order (ascending
// forward, descending backward), so a row waits only on rows of earlier tickets, held by blocks
// that already run; it polls the levels of its dependencies (sentinel -1, bounded wait) and
// publishes its own.  Rows are then ordered by level (counting sort; the order inside a level does
// not change any result, since rows of one level are independent) and the SELL-32 dependency
// tables are filled.
__global__ void __launch_bounds__(128) k_levels_sf(int32_t n, unsigned *ticket, const int32_t *__restrict__ rp,
                                                   const int32_t *__restrict__ ci, int32_t *lev, int forward,
                                                   int32_t *err) {
    __shared__ unsigned blk;
    const unsigned nchunks = (unsigned)((n + 127) / 128);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) blk = atomicAdd(ticket, 1u);
        __syncthreads();
        const unsigned b = blk;
        if (b >= nchunks) return;
        const int32_t t = (int32_t)(b * 128 + threadIdx.x);
        if (t >= n) continue;
        const int32_t i = forward ? t : n - 1 - t;
        const int32_t k0 = rp[i], k1 = rp[i + 1];
        int32_t l = 0;
        unsigned long long t0 = 0;
        for (int round = 0;; ++round) {
            bool pending = false;
            l = 0;
#pragma unroll 4
            for (int32_t k = k0; k < k1; ++k) {
                const int32_t j = ci[k];
                if (forward ? (j < i) : (j > i)) {
                    int32_t v;
                    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(lev + j) : "memory");
                    pending |= v < 0;
                    l = max(l, v + 1);
                }
            }
            if (!pending) break;
            if (round == 0) t0 = gtimer();
            else if (gtimer() - t0 > kWaitNs) { atomicExch(err, 1); break; }
            __nanosleep(20);
        }
        asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(lev + i), "r"(l) : "memory");
    }
}
__global__ void k_compose(int32_t n, const int32_t *a, const int32_t *b, int32_t *out) {  // out[t] = a[b[t]]
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = a[b[t]];
}
// dependency count of the row at each position -> per-chunk width (warp max)
__global__ void k_chunk_width(int32_t n, const int32_t *pos, const int32_t *rp, const int32_t *dg, int lower,
                              int32_t *w) {
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    int32_t cnt = 0;
    if (t < n) {
        int32_t row = pos[t];
        cnt = lower ? dg[row] - rp[row] : rp[row + 1] - dg[row] - 1;
    }
    cnt = __reduce_max_sync(0xffffffffu, cnt);
    if ((t & 31) == 0 && (t >> 5) < (n + 31) / 32) w[t >> 5] = cnt;
}
__global__ void k_widen(int32_t m, const int32_t *a, int64_t *b) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= m) b[i] = a[i];
}
__global__ void k_fill_tables(int32_t n, const int32_t *pos, const int32_t *rp, const int32_t *ci, const int32_t *dg,
                              const int32_t *inv, int lower, const int32_t *off, int32_t *col, int32_t *kidx) {
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int32_t row = pos[t], ch = t >> 5, lane = t & 31;
    int32_t k0 = lower ? rp[row] : dg[row] + 1, k1 = lower ? dg[row] : rp[row + 1];
    for (int32_t k = k0; k < k1; ++k) {
        int64_t u = ((int64_t)off[ch] + (k - k0)) * 32 + lane;
        col[u] = inv[ci[k]];
        kidx[u] = k;
    }
}
__global__ void k_dinv_index(int32_t n, const int32_t *pos_b, const int32_t *dg, int32_t *kidx) {
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) kidx[t] = dg[pos_b[t]];
}

// largest row length, lower count and upper count of a pattern (atomic maxima per warp)
__global__ void k_row_extents(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int32_t *ext) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    int32_t len = 0, lower = 0, upper = 0;
    if (i < n) {
        len = rp[i + 1] - rp[i];
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
            lower += ci[k] < i;
            upper += ci[k] > i;
        }
    }
    len = __reduce_max_sync(0xffffffffu, len);
    lower = __reduce_max_sync(0xffffffffu, lower);
    upper = __reduce_max_sync(0xffffffffu, upper);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(ext, len);
        atomicMax(ext + 1, lower);
        atomicMax(ext + 2, upper);
    }
}

// Block ILU(0) factorisation in one launch: rows in forward level order, taken in ticket order;
// a row waits (bounded) until every row it depends on has published its factored blocks
// (release store of its flag), then computes its own blocks as in the level-by-level form.
template <int B>
__global__ void __launch_bounds__(64) k_bilu_factor_sf(int32_t n, unsigned *ticket, const int32_t *__restrict__ pos,
                                                       const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                                       const int32_t *__restrict__ diag, double *LU, int32_t *flag,
                                                       int32_t epoch, int32_t *singular, KState *ks) {
    __shared__ unsigned blk;
    const unsigned nchunks = (unsigned)((n + 63) / 64);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) blk = atomicAdd(ticket, 1u);
        __syncthreads();
        const unsigned b = blk;
        if (b >= nchunks) return;
        const int32_t t = (int32_t)(b * 64 + threadIdx.x);
        if (t >= n) continue;
        const int32_t i = pos[t];
        const int32_t e = rp[i + 1];
        // wait until every row this row depends on has published its blocks: poll all flags
        // together, then re-poll only the ones not yet set
        {
            const int32_t k0 = rp[i], k1 = diag[i];
            unsigned long long t0 = 0;
            bool pending = true;
            for (int round = 0; pending; ++round) {
                pending = false;
                for (int32_t k = k0; k < k1; ++k) {
                    int32_t f;
                    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(f) : "l"(flag + ci[k]) : "memory");
                    pending |= f != epoch;
                }
                if (!pending) break;
                if (round == 0) t0 = gtimer();
                else if (gtimer() - t0 > kWaitNs) { atomicExch(&ks->wait_err, 1); break; }
                __nanosleep(20);
            }
        }
        for (int32_t k = rp[i]; k < diag[i]; ++k) {
            const int32_t c = ci[k];
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
                const int32_t j = ci[qq];
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
        if (!block_inverse<B>(d)) atomicOr(singular, 1);
#pragma unroll
        for (int q = 0; q < B * B; ++q) dd[q] = d[q];
        asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(flag + i), "r"(epoch) : "memory");
    }
}


// In-place inverse of the pivot block by the four lanes of a row's group, lane r holding row r of
// [D | I] (lanes r >= B only take part in the shuffles): Gauss-Jordan with partial pivoting, the
// same operations and order as block_inverse (largest |d_rk| among the remaining rows, lowest row
// on ties; the pivot row times 1 / pivot; every other row minus its multiple of the pivot row).
// The rows are not moved: each lane keeps the index of the row it holds.  The pivot search
// compares the bit patterns of |d_rk| as integers (for non-negative doubles their order is the
// numeric order), so it takes no turn on the FP64 pipe; a NaN candidate makes the block singular.
// Returns false if singular (the block is then left as it was).
constexpr long long kInfBits = 0x7ff0000000000000LL;   // bit pattern of +inf
template <int B>
__device__ __forceinline__ bool group_inverse(double *blk, int r, unsigned gmask, int g0) {
    double a[2 * B];
#pragma unroll
    for (int q = 0; q < B; ++q) a[q] = r < B ? blk[r * B + q] : 0.0;
#pragma unroll
    for (int q = 0; q < B; ++q) a[B + q] = (q == r) ? 1.0 : 0.0;
    int ri = r;
#pragma unroll
    for (int k = 0; k < B; ++k) {
        const bool cand = r < B && ri >= k;
        long long v = cand ? __double_as_longlong(fabs(a[k])) : -1LL;
        int idx = cand ? ri : 0x7fffffff;
#pragma unroll
        for (int o = 1; o < kSfGroup; o <<= 1) {
            const long long ov = __shfl_xor_sync(gmask, v, o);
            const int oi = __shfl_xor_sync(gmask, idx, o);
            if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
        }
        if (!(v > 0 && v <= kInfBits)) return false;
        const int p = idx;
        if (r < B) {
            if (ri == k) ri = p;
            else if (ri == p) ri = k;
        }
        const unsigned pl = __ballot_sync(gmask, r < B && ri == k);
        const int src = __ffs(pl) - 1;
        if (r < B && ri == k) {
            const double d = 1.0 / a[k];
#pragma unroll
            for (int q = 0; q < 2 * B; ++q) a[q] *= d;
        }
        double pr[2 * B];
#pragma unroll
        for (int q = 0; q < 2 * B; ++q) pr[q] = __shfl_sync(gmask, a[q], src);
        if (r < B && ri != k) {
            const double f = a[k];
#pragma unroll
            for (int q = 0; q < 2 * B; ++q) a[q] = fma(-f, pr[q], a[q]);
        }
    }
    __syncwarp(gmask);
    if (r < B)
#pragma unroll
        for (int q = 0; q < B; ++q) blk[ri * B + q] = a[B + q];
    (void)g0;
    return true;
}

// The same inverse by a whole warp, one lane per entry of [D | I]: lane s * 2B + q holds entry q of
// the row that started in slot s (2 B^2 lanes; the others only take part in the shuffles), and
// every lane keeps the positions of all B rows, updated alike.  Each entry gets the operations of
// block_inverse in the same order (the pivot row times 1 / pivot, every other row minus f times the
// scaled pivot row), so the inverse is the same bit for bit.  On GB300 a warp-wide FP64 instruction
// holds the sub-partition's pipe for 64 cycles: a step issues the reciprocal, one multiply and one
// FMA, against 2B multiplies and 2B FMAs with a row per lane.  Returns false if singular (the same in every
// lane; the block is then left as it was).
template <int B>
__device__ __forceinline__ bool warp_inverse(double *blk, int lane) {
    constexpr int W2 = 2 * B;
    constexpr unsigned kAll = 0xffffffffu;
    const bool act = lane < B * W2;
    const int s = act ? lane / W2 : 0, q = act ? lane - s * W2 : 0;
    double a = 0.0;
    if (act) a = q < B ? blk[s * B + q] : (q - B == s ? 1.0 : 0.0);
    int ri[B];
#pragma unroll
    for (int u = 0; u < B; ++u) ri[u] = u;
#pragma unroll
    for (int k = 0; k < B; ++k) {
        // largest |d_rk| among the rows at positions >= k, lowest position on ties
        const long long mine = __double_as_longlong(fabs(a));
        long long best = -1LL;
        int p = 0x7fffffff;
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const long long v = __shfl_sync(kAll, mine, u * W2 + k);
            if (ri[u] >= k && (v > best || (v == best && ri[u] < p))) { best = v; p = ri[u]; }
        }
        if (!(best > 0 && best <= kInfBits)) return false;
        int ps = 0;   // the slot whose row moves to position k
#pragma unroll
        for (int u = 0; u < B; ++u) {
            if (ri[u] == k) ri[u] = p;
            else if (ri[u] == p) ri[u] = k;
            if (ri[u] == k) ps = u;
        }
        const double d = 1.0 / __shfl_sync(kAll, a, ps * W2 + k);
        const double f = __shfl_sync(kAll, a, s * W2 + k);
        if (act && s == ps) a *= d;
        const double pr = __shfl_sync(kAll, a, ps * W2 + q);
        if (act && s != ps) a = fma(-f, pr, a);
    }
    int rs = 0;   // the final position of this lane's row (a select chain keeps ri in registers)
#pragma unroll
    for (int u = 0; u < B; ++u)
        if (u == s) rs = ri[u];
    __syncwarp();
    if (act && q >= B) blk[rs * B + (q - B)] = a;
    return true;
}

// The factorisation with a row over four lanes (B <= 4) and its memory traffic batched, so that
// once its last dependency is published a row costs one memory round trip before it computes.
// Before the flags are set (off the critical path, since tickets run levels ahead): the row's
// own blocks and columns, then the pivot and row-end positions of its dependencies, then the
// column indices of their upper parts, all by cp.async into shared memory (none of these are
// written during the launch).  Once every flag is set and acquire fences order what follows:
// each dependency's pivot inverse and upper blocks (one contiguous run of blocks) by 16-byte
// cp.async through L2 only, into a window rounded out to 16-byte boundaries (LU has two spare
// doubles for that).  Lane r then computes row r of every block of the row (its B FMAs per entry
// of L_ik = A_ik D_k^{-1} and of each update A_ij -= L_ik U_kj, in the order of
// k_bilu_factor_sf), and the four lanes invert the pivot block together (group_inverse).  The
// pivot and upper blocks are written and the flag released before the lower blocks are written
// (no row of the launch reads those).  Shared memory per row: rowsz doubles for the row's blocks
// (even), maxdep windows of W doubles, and maxrow + 2 maxdep + maxdep maxu integers; kSfRowsG
// rows per block.  Patterns too wide for that run k_bilu_factor_sf.
template <int B>
__global__ void __launch_bounds__(kSfThreads) k_bilu_factor_g(int32_t n, unsigned *ticket, const int32_t *__restrict__ pos,
                                                             const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                                             const int32_t *__restrict__ diag, double *LU, int32_t *flag,
                                                             int32_t epoch, int32_t *singular, KState *ks, int maxrow,
                                                             int maxdep, int maxu) {
    constexpr int BB = B * B, G = kSfGroup;
    extern __shared__ __align__(16) unsigned char fs_smem[];
    const int rowsz = (maxrow * BB + 1) & ~1;
    const int W = ((1 + maxu) * BB + 2 + 1) & ~1;
    const int per = rowsz + maxdep * W;
    const int j = threadIdx.x / G, r = threadIdx.x & (G - 1);
    const int g0 = (threadIdx.x & 31) & ~(G - 1);
    const unsigned gmask = 0xFu << g0;
    double *rowb = reinterpret_cast<double *>(fs_smem) + (int64_t)j * per;
    double *depw = rowb + rowsz;
    const int iper = maxrow + maxdep * (2 + maxu);
    int32_t *cols = reinterpret_cast<int32_t *>(reinterpret_cast<double *>(fs_smem) + (int64_t)kSfRowsG * per) + j * iper;
    int32_t *dcs = cols + maxrow, *ecs = dcs + maxdep, *ucol = ecs + maxdep;
    __shared__ unsigned blk;
    const unsigned nchunks = (unsigned)((n + kSfRowsG - 1) / kSfRowsG);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) blk = atomicAdd(ticket, 1u);
        __syncthreads();
        const unsigned b = blk;
        if (b >= nchunks) return;
        const int32_t t = (int32_t)(b * kSfRowsG + j);
        bool done = t >= n;                         // the whole group
        int32_t i = 0, k0 = 0, e = 0, kd = 0, len = 0, nd = 0;
        if (!done) {
            i = pos[t];
            k0 = rp[i];
            e = rp[i + 1];
            kd = diag[i];
            len = e - k0;
            nd = kd - k0;
            for (int32_t k = r; k < len; k += G) cp_async_i32(cols + k, ci + k0 + k);
            cp_async_commit();
            for (int32_t u = r; u < len * BB; u += G) cp_async_elem(rowb + u, LU + (int64_t)k0 * BB + u);
            cp_async_commit();
            cp_async_wait_1();
            __syncwarp(gmask);
            for (int32_t k = r; k < nd; k += G) {
                const int32_t c = cols[k];
                cp_async_i32(dcs + k, diag + c);
                cp_async_i32(ecs + k, rp + c + 1);
            }
            cp_async_commit();
            cp_async_wait_0();
            __syncwarp(gmask);
            for (int32_t k = 0; k < nd; ++k)
                for (int32_t qq = dcs[k] + 1 + r; qq < ecs[k]; qq += G)
                    cp_async_i32(ucol + k * maxu + (qq - dcs[k] - 1), ci + qq);
            cp_async_commit();
        }
        // Lockstep rounds over the warp (as in the sweeps): every unfinished group reads its
        // dependency flags once per round; the groups whose flags are all set factor their rows
        // in that round, together.  No group waits for another one.
        unsigned long long t0 = 0;
        bool waiting = false;
        while (__any_sync(0xffffffffu, !done)) {
            bool pend = false;
            if (!done) {
                bool p = false;   // the four lanes of the row poll a quarter of the flags each
                for (int32_t k = r; k < nd; k += G) {
                    int32_t f;
                    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(f) : "l"(flag + cols[k]) : "memory");
                    p |= f != epoch;
                }
                p = __any_sync(gmask, p);
                if (p) {
                    bool late = false;
                    if (!waiting) {
                        t0 = gtimer();
                        waiting = true;
                    } else {
                        late = gtimer() - t0 > kWaitNs;
                    }
                    if (__any_sync(gmask, late)) {
                        if (r == 0) atomicExch(&ks->wait_err, 1);
                        p = false;
                    } else {
                        pend = true;
                    }
                }
                if (!p) {
                    // each lane's acquire loads order what follows after the flags it read; the warp
                    // barrier then orders every lane's copies after all four lanes' acquires
                    __syncwarp(gmask);
                    for (int32_t k = 0; k < nd; ++k) {
                        const int64_t lo = (int64_t)dcs[k] * BB, hi = (int64_t)ecs[k] * BB;
                        const int64_t a0 = lo & ~(int64_t)1;
                        double *w = depw + (int64_t)k * W;
                        for (int64_t u = a0 + 2 * r; u < hi; u += 2 * G) cp_async_cg16(w + (u - a0), LU + u);
                    }
                    cp_async_commit();
                    cp_async_wait_0();
                    __syncwarp(gmask);
                    if (r < B) {
                        for (int32_t k = k0; k < kd; ++k) {
                            const int32_t dc = dcs[k - k0], ec = ecs[k - k0];
                            const double *dinv = depw + (int64_t)(k - k0) * W + (int)(((int64_t)dc * BB) & 1);
                            const int32_t *uc = ucol + (k - k0) * maxu;
                            double a[B], l[B];
#pragma unroll
                            for (int q = 0; q < B; ++q) a[q] = rowb[(k - k0) * BB + r * B + q];
#pragma unroll
                            for (int q = 0; q < B; ++q) {
                                double sacc = 0.0;
#pragma unroll
                                for (int u = 0; u < B; ++u) sacc = fma(a[u], dinv[u * B + q], sacc);
                                l[q] = sacc;
                            }
#pragma unroll
                            for (int q = 0; q < B; ++q) rowb[(k - k0) * BB + r * B + q] = l[q];
                            int32_t p2 = k + 1;
                            for (int32_t qq = dc + 1; qq < ec; ++qq) {
                                const int32_t jj = uc[qq - dc - 1];
                                while (p2 < e && cols[p2 - k0] < jj) ++p2;
                                if (p2 < e && cols[p2 - k0] == jj) {
                                    const double *u = dinv + (qq - dc) * BB;
                                    double *d = rowb + (p2 - k0) * BB + r * B;
#pragma unroll
                                    for (int q = 0; q < B; ++q) {
                                        double sacc = d[q];
#pragma unroll
                                        for (int w2 = 0; w2 < B; ++w2) sacc = fma(-l[w2], u[w2 * B + q], sacc);
                                        d[q] = sacc;
                                    }
                                }
                            }
                        }
                    }
                    __syncwarp(gmask);
                    if (!group_inverse<B>(rowb + nd * BB, r, gmask, g0) && r == 0) atomicOr(singular, 1);
                    __syncwarp(gmask);
                    for (int32_t u = nd * BB + r; u < len * BB; u += G) LU[(int64_t)k0 * BB + u] = rowb[u];
                    // the warp barrier orders the four lanes' stores before lane 0's release store,
                    // which publishes them all (release is cumulative)
                    __syncwarp(gmask);
                    if (r == 0) asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(flag + i), "r"(epoch) : "memory");
                    for (int32_t u = r; u < nd * BB; u += G) LU[(int64_t)k0 * BB + u] = rowb[u];
                    done = true;
                }
            }
            if (__any_sync(0xffffffffu, pend)) __nanosleep(20);
        }
    }
}

// The factorisation with a row per warp.  On GB300 a warp-wide FP64 instruction occupies a
// sub-partition's FP64 pipe for 64 cycles, so a level's time is bounded by the FP64 instructions
// the warp holding a row issues: here every block product is spread over the lanes (one lane per
// entry of L_ik = A_ik D_k^{-1}, one per entry of each updated block A_ij -= L_ik U_kj: six FP64
// instructions per dependency of a 3 x 3 row), and so is the pivot inverse (warp_inverse: per
// pivot step a reciprocal, one multiply and one FMA).  Each entry is summed in the order of
// k_bilu_factor_sf (the same values).  Warps take rows by ticket in level order, so every
// dependency belongs to a warp that is already running.  Before the flags are set: the row's own
// blocks and columns, the pivot and row-end positions of its dependencies and the column indices
// of their upper parts (none written during the launch).  Once every flag is set and an acquire
// fence orders what follows: each dependency's pivot inverse and upper blocks, read through L2.
// The pivot and upper blocks are written and the flag released before the lower blocks (no row of
// the launch reads those).  Shared memory per warp: the row's blocks, the dependencies' windows,
// L_ik, and the integer tables (kFwWarps warps per block).
constexpr int kFwWarps = 4;
__host__ __device__ inline int fw_row_doubles(int B, int maxrow) { return (maxrow * B * B + 1) & ~1; }
__host__ __device__ inline int fw_win_doubles(int B, int maxu) { return ((1 + maxu) * B * B + 1) & ~1; }
__host__ __device__ inline int fw_warp_doubles(int B, int maxrow, int maxdep, int maxu) {
    return fw_row_doubles(B, maxrow) + maxdep * fw_win_doubles(B, maxu) + ((B * B + 1) & ~1);
}
__host__ __device__ inline int fw_warp_ints(int maxrow, int maxdep, int maxu) {
    return maxrow + maxdep * (2 + maxu) + maxu;
}

template <int B>
__global__ void __launch_bounds__(32 * kFwWarps) k_bilu_factor_w(int32_t n, unsigned *ticket,
                                                                 const int32_t *__restrict__ pos,
                                                                 const int32_t *__restrict__ rp,
                                                                 const int32_t *__restrict__ ci,
                                                                 const int32_t *__restrict__ diag, double *LU,
                                                                 int32_t *flag, int32_t epoch, int32_t *singular,
                                                                 KState *ks, int maxrow, int maxdep, int maxu) {
    constexpr int BB = B * B;
    constexpr unsigned kAll = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char fw_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per = fw_warp_doubles(B, maxrow, maxdep, maxu), W = fw_win_doubles(B, maxu);
    double *rowb = reinterpret_cast<double *>(fw_smem) + (int64_t)warp * per;
    double *depw = rowb + fw_row_doubles(B, maxrow);
    double *lbuf = depw + (int64_t)maxdep * W;
    int32_t *cols = reinterpret_cast<int32_t *>(reinterpret_cast<double *>(fw_smem) + (int64_t)kFwWarps * per) +
                    warp * fw_warp_ints(maxrow, maxdep, maxu);
    int32_t *dcs = cols + maxrow, *ecs = dcs + maxdep, *ucol = ecs + maxdep, *upos = ucol + maxdep * maxu;
    for (;;) {
        unsigned tk = 0;
        if (lane == 0) tk = atomicAdd(ticket, 1u);
        const int32_t t = (int32_t)__shfl_sync(kAll, tk, 0);
        if (t >= n) return;
        const int32_t i = pos[t], k0 = rp[i], e = rp[i + 1], kd = diag[i];
        const int32_t len = e - k0, nd = kd - k0;
        for (int32_t k = lane; k < len; k += 32) cols[k] = (int32_t)chk(ci[k0 + k], n, CHK_FACTOR_COL);
        for (int32_t u = lane; u < len * BB; u += 32) rowb[u] = LU[(int64_t)k0 * BB + u];
        __syncwarp();
        for (int32_t k = lane; k < nd; k += 32) {
            const int32_t c = cols[k];
            dcs[k] = (int32_t)chk(diag[c], rp[n], CHK_FACTOR_DEP);
            ecs[k] = rp[c + 1];
        }
        __syncwarp();
        for (int32_t k = 0; k < nd; ++k)
            for (int32_t qq = dcs[k] + 1 + lane; qq < ecs[k]; qq += 32)
                ucol[k * maxu + (qq - dcs[k] - 1)] = (int32_t)chk(ci[qq], n, CHK_FACTOR_COL);
        // the dependencies' flags (each lane polls some), bounded
        unsigned long long tw = 0;
        bool waiting = false;
        for (;;) {
            bool p = false;
            for (int32_t k = lane; k < nd; k += 32) {
                int32_t f;
                asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(f) : "l"(flag + cols[k]) : "memory");
                p |= f != epoch;
            }
            if (!__any_sync(kAll, p)) break;
            bool late = false;
            if (!waiting) {
                tw = gtimer();
                waiting = true;
            } else {
                late = gtimer() - tw > kWaitNs;
            }
            if (__any_sync(kAll, late)) {
                if (lane == 0) atomicExch(&ks->wait_err, 1);
                break;
            }
            __nanosleep(20);
        }
        // each lane's acquire loads order its later reads after the flags it saw; the warp barrier
        // orders every lane's reads after all lanes' acquires
        __syncwarp();
        for (int32_t k = 0; k < nd; ++k) {
            const int64_t lo = (int64_t)dcs[k] * BB, hi = (int64_t)ecs[k] * BB;
            for (int64_t u = lo + lane; u < hi; u += 32) depw[(int64_t)k * W + (u - lo)] = __ldcg(LU + u);
        }
        __syncwarp();
        for (int32_t k = 0; k < nd; ++k) {
            const double *dinv = depw + (int64_t)k * W;   // the pivot inverse, then the upper blocks
            const int32_t m = ecs[k] - dcs[k] - 1;
            for (int32_t q2 = lane; q2 < m; q2 += 32) {   // where each upper block of row k sits in row i
                const int32_t jj = ucol[k * maxu + q2];
                int32_t p = -1;
                for (int32_t c = k + 1; c < len; ++c)
                    if (cols[c] == jj) {
                        p = c;
                        break;
                    }
                upos[q2] = p;
            }
            if (lane < BB) {   // L_ik = A_ik D_k^{-1}
                const int rr = lane / B, q = lane - rr * B;
                double sacc = 0.0;
#pragma unroll
                for (int u = 0; u < B; ++u) sacc = fma(rowb[k * BB + rr * B + u], dinv[u * B + q], sacc);
                lbuf[lane] = sacc;
            }
            __syncwarp();
            if (lane < BB) rowb[k * BB + lane] = lbuf[lane];
            for (int32_t x = lane; x < m * BB; x += 32) {   // A_ij -= L_ik U_kj
                const int32_t q2 = x / BB, ee = x - q2 * BB;
                const int32_t p = upos[q2];
                if (p >= 0) {
                    const int rr = ee / B, q = ee - rr * B;
                    const double *u = dinv + (q2 + 1) * BB;
                    double sacc = rowb[p * BB + ee];
#pragma unroll
                    for (int w2 = 0; w2 < B; ++w2) sacc = fma(-lbuf[rr * B + w2], u[w2 * B + q], sacc);
                    rowb[p * BB + ee] = sacc;
                }
            }
            __syncwarp();
        }
        if (!warp_inverse<B>(rowb + nd * BB, lane) && lane == 0) atomicOr(singular, 1);
        __syncwarp();
        for (int32_t u = nd * BB + lane; u < len * BB; u += 32) LU[(int64_t)k0 * BB + u] = rowb[u];
        // the warp barrier orders every lane's stores before lane 0's release store, which
        // publishes them all (release is cumulative)
        __syncwarp();
        if (lane == 0) asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(flag + i), "r"(epoch) : "memory");
        for (int32_t u = lane; u < nd * BB; u += 32) LU[(int64_t)k0 * BB + u] = rowb[u];
        __syncwarp();
    }
}

// level sets of one direction: pos (position -> row), inv, and the level pointers (host)
// stable counting sort of the rows by level on the host (rows of a level in ascending order keep
// the sweeps' accesses local): positions -> rows, rows -> positions, level pointers
static void sort_by_level(int32_t n, const std::vector<int32_t> &hl, std::vector<int32_t> &hp, std::vector<int32_t> &hi,
                          std::vector<int32_t> &h_lptr) {
    int32_t nl = 0;
    for (int32_t i = 0; i < n; ++i) nl = std::max(nl, hl[i] + 1);
    h_lptr.assign(nl + 1, 0);
    for (int32_t i = 0; i < n; ++i) h_lptr[hl[i] + 1]++;
    for (int32_t l = 0; l < nl; ++l) h_lptr[l + 1] += h_lptr[l];
    std::vector<int32_t> cur(h_lptr.begin(), h_lptr.end() - 1);
    hp.resize(n);
    hi.resize(n);
    for (int32_t i = 0; i < n; ++i) {
        int32_t t = cur[hl[i]]++;
        hp[t] = i;
        hi[i] = t;
    }
}

// level sets of both sweeps: the forward levels on the main stream and the backward ones on the
// side stream at the same time (both launches are latency bound), then the two sorts
static cptr_status device_levels(Ctx *c, const int32_t *rp, const int32_t *ci, int32_t *pos_f, int32_t *inv_f,
                                 std::vector<int32_t> &lptr_f, int32_t *pos_b, int32_t *inv_b,
                                 std::vector<int32_t> &lptr_b, int32_t *levr_f, int32_t *levr_b) {
    const int32_t n = c->n;
    cudaStream_t s = c->stream;
    if (!c->side_stream) CPTR_CUDA_TRY(c, cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking));
    if (!c->side_fork) CPTR_CUDA_TRY(c, cudaEventCreateWithFlags(&c->side_fork, cudaEventDisableTiming));
    if (!c->side_join) CPTR_CUDA_TRY(c, cudaEventCreateWithFlags(&c->side_join, cudaEventDisableTiming));
    int32_t *lev = nullptr, *tk = nullptr;
    CPTR_TRY(dalloc_t(c, &lev, 2 * (size_t)n));
    CPTR_TRY(dalloc_t(c, &tk, 4));   // ticket and wait error of each direction
    CPTR_CUDA_TRY(c, cudaMemsetAsync(lev, 0xFF, sizeof(int32_t) * 2 * (size_t)n, s));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(tk, 0, 4 * sizeof(int32_t), s));
    CPTR_CUDA_TRY(c, cudaEventRecord(c->side_fork, s));
    CPTR_CUDA_TRY(c, cudaStreamWaitEvent(c->side_stream, c->side_fork, 0));
    const unsigned grid = std::min<unsigned>(nblk(n, 128), 8 * 152);
    (k_levels_sf<<<grid, 128, 0, s>>>(n, reinterpret_cast<unsigned *>(tk), rp, ci, lev, 1, tk + 1), note_launch());
    (k_levels_sf<<<grid, 128, 0, c->side_stream>>>(n, reinterpret_cast<unsigned *>(tk + 2), rp, ci, lev + n, 0, tk + 3),
     note_launch());
    CPTR_CUDA_TRY(c, cudaGetLastError());
    CPTR_CUDA_TRY(c, cudaEventRecord(c->side_join, c->side_stream));
    CPTR_CUDA_TRY(c, cudaStreamWaitEvent(s, c->side_join, 0));
    std::vector<int32_t> hl(2 * (size_t)n), hp, hi;
    int32_t werr[4] = {0, 0, 0, 0};
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(werr, tk, sizeof(werr), cudaMemcpyDeviceToHost, s));
    const cptr_status cs = copy_to_host(c, hl.data(), lev, sizeof(int32_t) * 2 * (size_t)n);
    dfree(tk);
    dfree(lev);
    CPTR_TRY(cs);
    if (werr[1] || werr[3]) return c->fail(CPTR_ETIMEOUT, "ILU(0) level sets: a bounded wait gave up");
    std::vector<int32_t> hlf(hl.begin(), hl.begin() + n), hlb(hl.begin() + n, hl.end());
    // the level of every row, for the paired-level tables
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(levr_f, hlf.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(levr_b, hlb.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    sort_by_level(n, hlf, hp, hi, lptr_f);
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(pos_f, hp.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(inv_f, hi.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(s));
    sort_by_level(n, hlb, hp, hi, lptr_b);
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(pos_b, hp.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(inv_b, hi.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(s));
    return CPTR_OK;
}

// SELL-32 dependency table of one sweep: chunk offsets (int64), dependency positions and the
// block index of every slot (-1 = padding)
static cptr_status device_table(Ctx *c, const int32_t *pos, const int32_t *inv, const int32_t *rp, const int32_t *ci,
                                const int32_t *dg, bool lower, int64_t **off64, int32_t **col, int32_t **kidx,
                                int64_t *nslots) {
    const int32_t n = c->n, nch = (n + 31) / 32;
    cudaStream_t s = c->stream;
    int32_t *w = nullptr, *off = nullptr;
    CPTR_TRY(dalloc_t(c, &w, (size_t)nch + 1));
    CPTR_TRY(dalloc_t(c, &off, (size_t)nch + 1));
    (k_chunk_width<<<nblk((int64_t)nch * 32, 256), 256, 0, s>>>(n, pos, rp, dg, lower ? 1 : 0, w), note_launch());
    int32_t total = 0;
    CPTR_TRY(scan_exclusive(c, w, off, nch, &total));
    CPTR_TRY(dalloc_t(c, off64, (size_t)nch + 1));
    (k_widen<<<nblk(nch + 1, 256), 256, 0, s>>>(nch, off, *off64), note_launch());
    const int64_t ns = (int64_t)total * 32;
    CPTR_TRY(dalloc_t(c, col, (size_t)(ns > 0 ? ns : 1)));
    CPTR_TRY(dalloc_t(c, kidx, (size_t)(ns > 0 ? ns : 1)));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(*col, 0xFF, sizeof(int32_t) * (ns > 0 ? ns : 1), s));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(*kidx, 0xFF, sizeof(int32_t) * (ns > 0 ? ns : 1), s));
    (k_fill_tables<<<nblk(n, 256), 256, 0, s>>>(n, pos, rp, ci, dg, inv, lower ? 1 : 0, off, *col, *kidx), note_launch());
    CPTR_CUDA_TRY(c, cudaGetLastError());
    dfree(w); dfree(off);
    *nslots = ns;
    return CPTR_OK;
}

// Greedy distance-1 colouring of the cell graph in natural order (smallest colour unused by the
// lower-index neighbours), cells sorted by (colour, index): new index -> original cell.
static std::vector<int32_t> multicolour_order(int32_t n, const std::vector<int32_t> &rp, const std::vector<int32_t> &ci) {
    std::vector<int32_t> color(n, 0), order;
    int32_t ncol = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t cc = 0;
        for (;;) {
            bool used = false;
            for (int32_t k = rp[i]; k < rp[i + 1] && !used; ++k) used = ci[k] < i && color[ci[k]] == cc;
            if (!used) break;
            ++cc;
        }
        color[i] = cc;
        ncol = std::max(ncol, cc + 1);
    }
    order.reserve(n);
    for (int32_t cc = 0; cc < ncol; ++cc)
        for (int32_t i = 0; i < n; ++i)
            if (color[i] == cc) order.push_back(i);
    return order;
}

__global__ void k_gather_blocks(int32_t nnzb, int BB, const int32_t *kmap, const double *src, double *dst) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= (int64_t)nnzb * BB) return;
    int64_t k = u / BB;
    int e = (int)(u % BB);
    dst[u] = src[(int64_t)kmap[k] * BB + e];
}

// Host tables of the chunked sweeps for one direction (forward: dependencies j < i, chunks in
// increasing order; backward: j > i, chunks in decreasing order).  Positions enumerate the rows
// chunk by chunk in processing order and, inside a chunk, by local level (rows in dependency
// order within a level).  code[d * n + p]: >= 0 a ring slot (local level mod W) * maxw + index in
// level; < 0 (but not kCwNone) the global row -(code + 1); kCwNone no dependency.  kidx gives the
// factor block of each slot (and, backward, the diagonal block in slot D).
struct CwHost {
    int32_t nchunks = 0, D = 0, W = 1, maxw = 0, nlev_total = 0, max_chunk_levels = 0;
    std::vector<int32_t> clev, lptr, prow, code, kidx;
};

// run f(c) for c in [0, count) on up to 16 host threads
template <typename F>
static void parallel_chunks(int32_t count, F &&f) {
    const int nt = (int)std::max(1u, std::min<unsigned>(8u, std::min<unsigned>(std::thread::hardware_concurrency(),
                                                                               (unsigned)count)));
    if (nt <= 1) {
        for (int32_t c = 0; c < count; ++c) f(c);
        return;
    }
    std::atomic<int32_t> next(0);
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t)
        pool.emplace_back([&]() {
            for (int32_t c = next++; c < count; c = next++) f(c);
        });
    for (auto &th : pool) th.join();
}

static CwHost cw_build(int32_t n, const std::vector<int32_t> &rp, const std::vector<int32_t> &ci,
                       const std::vector<int32_t> &dg, int32_t K, bool forward) {
    CwHost h;
    const int32_t nch = (n + K - 1) / K;
    h.nchunks = nch;
    std::vector<int32_t> lev(n, 0), idx(n, 0);
    auto is_dep = [forward](int32_t i, int32_t j) { return forward ? j < i : j > i; };
    auto chunk_of_t = [&](int32_t t) { return forward ? t : nch - 1 - t; };   // t: processing order
    std::vector<int32_t> nl(nch, 0), md(nch, 0), dd(nch, 0), mw(nch, 0);
    std::vector<std::vector<int32_t>> cnts(nch);
    // 1. local levels (dependencies inside the chunk), level sizes, largest in-chunk distance,
    //    dependency count
    parallel_chunks(nch, [&](int32_t t) {
        const int32_t c = chunk_of_t(t);
        const int32_t r0 = c * K, r1 = std::min<int32_t>(n, r0 + K);
        int32_t maxl = 0, D = 0, maxdist = 0;
        for (int32_t u = 0; u < r1 - r0; ++u) {
            const int32_t i = forward ? r0 + u : r1 - 1 - u;
            int32_t l = 0, nd = 0;
            for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
                const int32_t j = ci[k];
                if (!is_dep(i, j)) continue;
                ++nd;
                if (j >= r0 && j < r1) l = std::max(l, lev[j] + 1);
            }
            lev[i] = l;
            maxl = std::max(maxl, l);
            D = std::max(D, nd);
        }
        std::vector<int32_t> &cnt = cnts[t];
        cnt.assign(maxl + 2, 0);
        for (int32_t i = r0; i < r1; ++i) {
            ++cnt[lev[i] + 1];
            for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
                const int32_t j = ci[k];
                if (is_dep(i, j) && j >= r0 && j < r1) maxdist = std::max(maxdist, lev[i] - lev[j]);
            }
        }
        int32_t w = 0;
        for (int32_t l = 0; l <= maxl; ++l) w = std::max(w, cnt[l + 1]);
        for (int32_t l = 0; l <= maxl; ++l) cnt[l + 1] += cnt[l];
        nl[t] = maxl + 1;
        md[t] = maxdist;
        dd[t] = D;
        mw[t] = w;
    });
    int32_t maxdist = 0;
    for (int32_t t = 0; t < nch; ++t) {
        maxdist = std::max(maxdist, md[t]);
        h.D = std::max(h.D, dd[t]);
        h.max_chunk_levels = std::max(h.max_chunk_levels, nl[t]);
        h.maxw = std::max(h.maxw, mw[t]);
    }
    h.W = std::min(maxdist, 3) + 1;
    // 2. offsets of every chunk's positions and levels (processing order)
    std::vector<int32_t> pos0(nch + 1, 0);
    h.clev.assign(nch + 1, 0);
    for (int32_t t = 0; t < nch; ++t) {
        const int32_t c = chunk_of_t(t);
        pos0[t + 1] = pos0[t] + (std::min<int32_t>(n, (c + 1) * K) - c * K);
        h.clev[t + 1] = h.clev[t] + nl[t];
    }
    h.nlev_total = h.clev[nch];
    h.lptr.assign((size_t)h.nlev_total + 1, n);
    h.prow.resize(n);
    const int nslots = h.D + (forward ? 0 : 1);
    h.code.assign((size_t)std::max(h.D, 1) * n, kCwNone);
    h.kidx.assign((size_t)std::max(nslots, 1) * n, -1);
    // 3. per chunk: stable counting sort by local level, then dependency codes and block indices
    parallel_chunks(nch, [&](int32_t t) {
        const int32_t c = chunk_of_t(t);
        const int32_t r0 = c * K, r1 = std::min<int32_t>(n, r0 + K);
        const std::vector<int32_t> &cnt = cnts[t];
        for (int32_t l = 0; l < nl[t]; ++l) h.lptr[h.clev[t] + l] = pos0[t] + cnt[l];
        std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
        for (int32_t u = 0; u < r1 - r0; ++u) {
            const int32_t i = forward ? r0 + u : r1 - 1 - u;
            const int32_t q = fill[lev[i]]++;
            h.prow[pos0[t] + q] = i;
            idx[i] = q - cnt[lev[i]];
        }
        for (int32_t p = pos0[t]; p < pos0[t + 1]; ++p) {
            const int32_t i = h.prow[p];
            int d = 0;
            for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
                const int32_t j = ci[k];
                if (!is_dep(i, j)) continue;
                const bool ring = j >= r0 && j < r1 && lev[i] - lev[j] <= h.W - 1;
                h.code[(size_t)d * n + p] = ring ? (lev[j] % h.W) * h.maxw + idx[j] : -(j + 1);
                h.kidx[(size_t)d * n + p] = k;
                ++d;
            }
            if (!forward) h.kidx[(size_t)h.D * n + p] = dg[i];
        }
    });
    return h;
}

// chunked tables of both sweeps (natural order only); c->cw_ok tells whether they fit
static cptr_status cw_setup(Ctx *c) {
    c->cw_ok = false;
    const int32_t n = c->n, B = c->b, BB = B * B;
    CPTR_TRY(host_pattern(c));
    const std::vector<int32_t> &rp = c->h_rp, &ci = c->h_ci;
    int32_t K = 1;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) K = std::max(K, std::abs(i - ci[k]));
    K = std::max<int32_t>(K, std::min<int32_t>(n, 4096));
    CwHost hf = cw_build(n, rp, ci, c->h_diag, K, true);
    CwHost hb = cw_build(n, rp, ci, c->h_diag, K, false);
    const bool lo = c->o.precision == CPTR_PREC_MIXED;
    const size_t tsz = lo ? 4 : 8;
    const int maxw = std::max(hf.maxw, hb.maxw);
    const int threads = std::max(32, (maxw + 31) / 32 * 32);
    const size_t rsz = 8;   // right-hand sides: FP64, or FP32 when the FP32 sweeps get FP32 input
    auto smem = [&](const CwHost &h, int extra, int S) {
        const size_t SW = (size_t)h.D * BB + extra;
        return cw_align16(tsz * h.W * h.maxw * B) + cw_align16(tsz * (S + 1) * threads * SW) +
               cw_align16((size_t)32 * (S + 1) * threads * h.D) + cw_align16(rsz * (S + 1) * threads * B) +
               cw_align16(4 * (size_t)(2 * S + 1) * threads) + cw_align16(4 * (size_t)(2 * S + 1) * h.D * threads) +
               (size_t)(h.max_chunk_levels + 1) * 4;
    };
    const size_t kLimit = 220 * 1024;
    // pipeline slack: 3 levels when it fits, else 2, else 1
    auto pick_s = [&](const CwHost &h, int extra) {
        for (int S : {3, 2, 1})
            if (smem(h, extra, S) <= kLimit) return S;
        return 0;
    };
    const int s_f = pick_s(hf, 0), s_b = pick_s(hb, BB);
    if (hf.D > kCwMaxD || hb.D > kCwMaxD || threads > kCwMaxThreads || s_f == 0 || s_b == 0) return CPTR_OK;
    cudaStream_t st = c->stream;
    auto up = [&](const std::vector<int32_t> &v, int32_t **dst) -> cptr_status {
        CPTR_TRY(dalloc_t(c, dst, std::max<size_t>(v.size(), 1)));
        if (!v.empty())
            CPTR_CUDA_TRY(c, cudaMemcpyAsync(*dst, v.data(), sizeof(int32_t) * v.size(), cudaMemcpyHostToDevice, st));
        return CPTR_OK;
    };
    CwTables *T2[2] = {&c->cw_f, &c->cw_b};
    const CwHost *H2[2] = {&hf, &hb};
    for (int dir = 0; dir < 2; ++dir) {
        CwTables &t = *T2[dir];
        const CwHost &h = *H2[dir];
        t.nchunks = h.nchunks;
        t.D = h.D;
        t.W = h.W;
        t.maxw = h.maxw;
        t.threads = threads;
        t.ns = dir ? s_b : s_f;   // pipeline slack S
        t.maxlev = h.max_chunk_levels;
        t.smem = (int32_t)smem(h, dir ? BB : 0, t.ns);
        CPTR_TRY(up(h.clev, &t.clev));
        CPTR_TRY(up(h.lptr, &t.lptr));
        CPTR_TRY(up(h.prow, &t.prow));
        CPTR_TRY(up(h.code, &t.code));
        CPTR_TRY(dalloc_t(c, &t.started, (size_t)std::max(h.nchunks, 1)));
        int32_t *kidx = nullptr;
        CPTR_TRY(up(h.kidx, &kidx));
        const int nslots = h.D + dir;
        CPTR_TRY(dalloc(c, &t.val, (size_t)std::max(nslots, 1) * BB * n * tsz));
        if (nslots > 0) {
            if (lo) (k_cw_pack<float><<<nblk((int64_t)nslots * n, 256), 256, 0, st>>>(n, nslots, BB, kidx, c->LU, (float *)t.val), note_launch());
            else (k_cw_pack<double><<<nblk((int64_t)nslots * n, 256), 256, 0, st>>>(n, nslots, BB, kidx, c->LU, (double *)t.val), note_launch());
        }
        CPTR_CUDA_TRY(c, cudaStreamSynchronize(st));
        dfree(kidx);
    }
    c->cw_ok = true;
    c->cw_use = c->o.ilu_sweep == 2;   // with autotune, the timing decides
    return CPTR_OK;
}

static void cw_free(Ctx *c) {
    for (CwTables *t : {&c->cw_f, &c->cw_b}) {
        dfree(t->clev); dfree(t->lptr); dfree(t->prow); dfree(t->code); dfree(t->val); dfree(t->started);
        *t = CwTables();
    }
    c->cw_ok = false;
    c->cw_use = false;
}

// ------------------------------------------------------------------------------------------------
// Grouped-level tables.  The levels of a sweep (its own level numbering) are taken in groups of G
// consecutive levels, [G0, G0 + G), solved as one step: a row of the group substitutes, along every
// chain of dependencies inside its group, the equations of those rows, so that it depends only on
// rows of earlier groups and on right-hand-side values.  G = 2 is the paired-level schedule (a row
// of odd level replaces its dependencies of the level before); G = 3 cuts the chain of dependent
// steps to a third.  With F_ik the factor of a dependency k of row i (forward L_ik; backward
// U_ik D_k^{-1} for k inside the group, U_ik for k outside, D_k^{-1} the stored inverted pivot):
//   forward, y = L^{-1} r:   y_i = c_i - sum_j M_ij y_j,         c_i = r_i - sum_l W_il r_l
//   backward, z = U^{-1} y:   z_i = D_i^{-1} (c_i - sum_j M_ij z_j), c_i = y_i - sum_l W_il y_l
// with, over the dependencies k of row i,
//   M_ij = [j outside the group] F_ij - sum_{k inside} F_ik M_kj,
//   W_il = [l inside the group] F_il - sum_{k inside} F_ik W_kl,
// M_kj and W_kl being row k's own expansion (a row at the group's first level keeps its own
// entries and has no W terms).  Mathematically these are the same solves; the sums are grouped
// differently, so values differ from the level-set sweeps by rounding only.  The tables are built
// in G passes, one per position in the group, each reading the expansions of the earlier positions.
// A row's M entries are ordered by dependency position, its W terms by first discovery in a
// depth-first walk of its in-group chains (the row's pattern order at every node); each entry
// starts from the row's own block (or zero) and subtracts the products in the row's pattern order.
constexpr int kPairMax = 32;   // entries of an expanded row; more and the tables are not built
constexpr int kGroupMax = 4;   // levels per group
constexpr int kInMax = 8;      // dependencies of a row inside its group; more and the tables are not built

// the dependencies of row u on the sweep's side of the diagonal: [*k0, *k1)
__device__ __forceinline__ void side_range(int lower, const int32_t *__restrict__ rp, const int32_t *__restrict__ dg,
                                           int32_t u, int32_t *k0, int32_t *k1) {
    *k0 = lower ? rp[u] : dg[u] + 1;
    *k1 = lower ? dg[u] : rp[u + 1];
}

// the distinct outside dependencies (as positions, J) and in-group sources (C, as source indices)
// reached from row i through chains inside its group; false if either exceeds kPairMax
__device__ bool group_sets(int32_t i, int32_t G0, int lower, const int32_t *__restrict__ inv,
                           const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const int32_t *__restrict__ dg, const int32_t *__restrict__ levr,
                           const int32_t *__restrict__ src_of_row, int32_t *J, int *nj, int32_t *C, int *nc) {
    int32_t node[kGroupMax], e[kGroupMax], e1[kGroupMax];
    int sp = 0;
    node[0] = i;
    side_range(lower, rp, dg, i, &e[0], &e1[0]);
    *nj = *nc = 0;
    bool ok = true;
    while (sp >= 0) {
        if (e[sp] == e1[sp]) {
            --sp;
            continue;
        }
        const int32_t k = ci[e[sp]++];
        if (levr[k] < G0) {
            const int32_t p = inv[k];
            bool seen = false;
            for (int q = 0; q < *nj; ++q) seen |= J[q] == p;
            if (!seen) {
                if (*nj == kPairMax) ok = false;
                else J[(*nj)++] = p;
            }
        } else {
            const int32_t l = src_of_row ? src_of_row[k] : k;
            bool seen = false;
            for (int q = 0; q < *nc; ++q) seen |= C[q] == l;
            if (!seen) {
                if (*nc == kPairMax) ok = false;
                else C[(*nc)++] = l;
            }
            if (sp + 1 < kGroupMax) {   // a chain inside the group is at most G - 1 links long
                ++sp;
                node[sp] = k;
                side_range(lower, rp, dg, k, &e[sp], &e1[sp]);
            } else {
                ok = false;
            }
        }
    }
    return ok;
}

// entry counts per position (main and W terms); *err set when a row exceeds kPairMax
__global__ void k_group_count(int32_t n, const int32_t *__restrict__ pos, const int32_t *__restrict__ inv,
                              const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              const int32_t *__restrict__ dg, const int32_t *__restrict__ levr, int lower, int G,
                              const int32_t *__restrict__ src_of_row, int32_t *mcnt, int32_t *ccnt, int32_t *err) {
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int32_t i = pos[t];
    const int32_t L = levr[i], G0 = L - L % G;
    if (L == G0) {   // the group's first level: the row's own entries
        int32_t k0, k1;
        side_range(lower, rp, dg, i, &k0, &k1);
        mcnt[t] = k1 - k0;
        ccnt[t] = 0;
        return;
    }
    int32_t J[kPairMax], C[kPairMax];
    int nj, nc;
    if (!group_sets(i, G0, lower, inv, rp, ci, dg, levr, src_of_row, J, &nj, C, &nc)) atomicExch(err, 1);
    int32_t k0, k1, nin = 0;
    side_range(lower, rp, dg, i, &k0, &k1);
    for (int32_t k = k0; k < k1; ++k) nin += levr[ci[k]] >= G0 ? 1 : 0;
    if (nin > kInMax) atomicExch(err, 1);
    mcnt[t] = nj;
    ccnt[t] = nc;
}

// the factor of dependency k of row i (entry e of the pattern): L_ik, U_ik, or U_ik D_k^{-1}
template <int B>
__device__ __forceinline__ void group_factor(const double *__restrict__ LU, int32_t e, int32_t dk, bool times_dinv,
                                             double *f) {
    constexpr int BB = B * B;
    if (!times_dinv) {
        for (int q = 0; q < BB; ++q) f[q] = LU[(int64_t)e * BB + q];
        return;
    }
    for (int r = 0; r < B; ++r)
        for (int q = 0; q < B; ++q) {
            double a = 0.0;
            for (int u = 0; u < B; ++u) a = fma(LU[(int64_t)e * BB + r * B + u], LU[(int64_t)dk * BB + u * B + q], a);
            f[r * B + q] = a;
        }
}
// m -= f * blk (B x B)
template <int B>
__device__ __forceinline__ void sub_product(double *m, const double *f, const double *__restrict__ blk) {
    for (int r = 0; r < B; ++r)
        for (int q = 0; q < B; ++q) {
            double a = m[r * B + q];
            for (int u = 0; u < B; ++u) a = fma(-f[r * B + u], blk[u * B + q], a);
            m[r * B + q] = a;
        }
}

// the entries of the rows at position p of their group (pass p; earlier positions are filled)
template <int B>
__global__ void k_group_fill(int32_t n, const int32_t *__restrict__ pos, const int32_t *__restrict__ inv,
                             const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                             const int32_t *__restrict__ dg, const int32_t *__restrict__ levr, int lower, int G, int p,
                             const double *__restrict__ LU, const int32_t *__restrict__ src_of_row,
                             const int32_t *__restrict__ mcnt, const int32_t *__restrict__ ccnt,
                             const int32_t *__restrict__ moff, const int32_t *__restrict__ coff, int32_t *mdep,
                             double *mblk, int32_t *cdep, double *cblk) {
    constexpr int BB = B * B;
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int32_t i = pos[t];
    const int32_t L = levr[i], G0 = L - L % G;
    if (L - G0 != p) return;
    int32_t k0, k1;
    side_range(lower, rp, dg, i, &k0, &k1);
    if (p == 0) {
        int32_t o = moff[t];
        for (int32_t k = k0; k < k1; ++k, ++o) {
            mdep[o] = inv[ci[k]];
            for (int e = 0; e < BB; ++e) mblk[(int64_t)o * BB + e] = LU[(int64_t)k * BB + e];
        }
        return;
    }
    int32_t J[kPairMax], C[kPairMax];
    int nj, nc;
    group_sets(i, G0, lower, inv, rp, ci, dg, levr, src_of_row, J, &nj, C, &nc);
    for (int a = 1; a < nj; ++a) {   // ascending dependency positions
        const int32_t v = J[a];
        int q = a - 1;
        while (q >= 0 && J[q] > v) { J[q + 1] = J[q]; --q; }
        J[q + 1] = v;
    }
    // the factors F_ik of the dependencies inside the group, in pattern order (at most kInMax, which
    // the counting pass checked), each formed once
    int32_t tin[kInMax], sin[kInMax];
    double fin[kInMax][BB];
    int nin = 0;
    for (int32_t k = k0; k < k1 && nin < kInMax; ++k) {
        const int32_t cc = ci[k];
        if (levr[cc] < G0) continue;
        tin[nin] = inv[cc];
        sin[nin] = src_of_row ? src_of_row[cc] : cc;
        group_factor<B>(LU, k, dg[cc], !lower, fin[nin]);
        ++nin;
    }
    const int32_t mo = moff[t], co = coff[t];
    for (int q = 0; q < nj; ++q) {
        const int32_t j = J[q];
        double m[BB];
        for (int e = 0; e < BB; ++e) m[e] = 0.0;
        for (int32_t k = k0; k < k1; ++k)   // the row's own block of an outside dependency
            if (levr[ci[k]] < G0 && inv[ci[k]] == j)
                for (int e = 0; e < BB; ++e) m[e] = LU[(int64_t)k * BB + e];
        for (int a = 0; a < nin; ++a) {   // minus F_ik M_kj over the dependencies inside the group
            const int32_t tk = tin[a], o1 = moff[tk] + mcnt[tk];
            for (int32_t o = moff[tk]; o < o1; ++o)
                if (mdep[o] == j) sub_product<B>(m, fin[a], mblk + (int64_t)o * BB);
        }
        mdep[mo + q] = j;
        for (int e = 0; e < BB; ++e) mblk[(int64_t)(mo + q) * BB + e] = m[e];
    }
    for (int q = 0; q < nc; ++q) {
        const int32_t l = C[q];
        double w[BB];
        for (int e = 0; e < BB; ++e) w[e] = 0.0;
        for (int a = 0; a < nin; ++a)   // F_il for a direct dependency inside the group
            if (sin[a] == l)
                for (int e = 0; e < BB; ++e) w[e] = fin[a][e];
        for (int a = 0; a < nin; ++a) {   // minus F_ik W_kl
            const int32_t tk = tin[a], o1 = coff[tk] + ccnt[tk];
            for (int32_t o = coff[tk]; o < o1; ++o)
                if (cdep[o] == l) sub_product<B>(w, fin[a], cblk + (int64_t)o * BB);
        }
        cdep[co + q] = l;
        for (int e = 0; e < BB; ++e) cblk[(int64_t)(co + q) * BB + e] = w[e];
    }
}

// backward tables: every block of the expanded row i (M and W entries) left-multiplied by row i's
// inverted pivot, z_i = D_i^{-1} y_i - sum_l (D_i^{-1} W_il) y_l - sum_j (D_i^{-1} M_ij) z_j, so that
// the sweep starts from D_i^{-1} y_i (known before any wait) and needs no product after its waits
template <int B>
__global__ void k_group_fold(int32_t n, const int32_t *__restrict__ pos, const int32_t *__restrict__ dg,
                             const double *__restrict__ LU, const int32_t *__restrict__ mcnt,
                             const int32_t *__restrict__ ccnt, const int32_t *__restrict__ moff,
                             const int32_t *__restrict__ coff, double *mblk, double *cblk) {
    constexpr int BB = B * B;
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double *d = LU + (int64_t)dg[pos[t]] * BB;
    for (int side = 0; side < 2; ++side) {
        double *blk = side == 0 ? mblk + (int64_t)moff[t] * BB : cblk + (int64_t)coff[t] * BB;
        const int32_t cnt = side == 0 ? mcnt[t] : ccnt[t];
        for (int32_t e = 0; e < cnt; ++e, blk += BB) {
            double m[BB];
            for (int r = 0; r < B; ++r)
                for (int q = 0; q < B; ++q) {
                    double a = 0.0;
                    for (int u = 0; u < B; ++u) a = fma(d[r * B + u], blk[u * B + q], a);
                    m[r * B + q] = a;
                }
            for (int q = 0; q < BB; ++q) blk[q] = m[q];
        }
    }
}

// SELL-32 tables from per-position entry lists (counts, CSR offsets, dependencies, blocks)
__global__ void k_chunk_width_cnt(int32_t n, const int32_t *cnt, int32_t *w) {
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    int32_t v = t < n ? cnt[t] : 0;
    v = __reduce_max_sync(0xffffffffu, v);
    if ((t & 31) == 0 && (t >> 5) < (n + 31) / 32) w[t >> 5] = v;
}
__global__ void k_fill_sell_csr(int32_t n, const int32_t *cnt, const int32_t *csr_off, const int32_t *dep,
                                const int32_t *off, int32_t *col, int32_t *kidx) {
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int32_t ch = t >> 5, lane = t & 31;
    for (int32_t e = 0; e < cnt[t]; ++e) {
        const int64_t u = ((int64_t)off[ch] + e) * 32 + lane;
        col[u] = dep[csr_off[t] + e];
        kidx[u] = csr_off[t] + e;
    }
}
// SELL-32 layout of per-position entry lists: chunk offsets, the column of every slot and its
// entry index in the lists (-1 for padding); *ns_out slots in all
static cptr_status sell_layout(Ctx *c, const int32_t *cnt, const int32_t *csr_off, const int32_t *dep,
                               int64_t **off64, int32_t **col, int32_t **kidx, int64_t *ns_out) {
    const int32_t n = c->n, nch = (n + 31) / 32;
    cudaStream_t s = c->stream;
    int32_t *w = nullptr, *off = nullptr;
    CPTR_TRY(dalloc_t(c, &w, (size_t)nch + 1));
    CPTR_TRY(dalloc_t(c, &off, (size_t)nch + 1));
    (k_chunk_width_cnt<<<nblk((int64_t)nch * 32, 256), 256, 0, s>>>(n, cnt, w), note_launch());
    int32_t total = 0;
    CPTR_TRY(scan_exclusive(c, w, off, nch, &total));
    CPTR_TRY(dalloc_t(c, off64, (size_t)nch + 1));
    (k_widen<<<nblk(nch + 1, 256), 256, 0, s>>>(nch, off, *off64), note_launch());
    const int64_t ns = (int64_t)total * 32;
    CPTR_TRY(dalloc_t(c, col, (size_t)(ns > 0 ? ns : 1)));
    CPTR_TRY(dalloc_t(c, kidx, (size_t)(ns > 0 ? ns : 1)));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(*col, 0xFF, sizeof(int32_t) * (ns > 0 ? ns : 1), s));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(*kidx, 0xFF, sizeof(int32_t) * (ns > 0 ? ns : 1), s));
    (k_fill_sell_csr<<<nblk(n, 256), 256, 0, s>>>(n, cnt, csr_off, dep, off, *col, *kidx), note_launch());
    CPTR_CUDA_TRY(c, cudaGetLastError());
    dfree(w); dfree(off);
    *ns_out = ns;
    return CPTR_OK;
}
// the slots' blocks, in the sweeps' precision
static cptr_status sell_pack(Ctx *c, const int32_t *kidx, int64_t ns, const double *blk, void **val) {
    const bool lo = c->o.precision == CPTR_PREC_MIXED;   // blocks stored in FP32
    const int BB = c->b * c->b;
    cudaStream_t s = c->stream;
    CPTR_TRY(dalloc(c, val, (size_t)(ns > 0 ? ns : 1) * BB * (lo ? 4 : 8)));
    if (ns > 0 && lo) (k_sf_pack<float><<<nblk(ns, 256), 256, 0, s>>>(ns, BB, kidx, blk, (float *)*val), note_launch());
    else if (ns > 0) (k_sf_pack<double><<<nblk(ns, 256), 256, 0, s>>>(ns, BB, kidx, blk, (double *)*val), note_launch());
    CPTR_CUDA_TRY(c, cudaGetLastError());
    return CPTR_OK;
}
template <typename I>
static cptr_status dcopy(Ctx *c, I **dst, const I *src, size_t count) {
    CPTR_TRY(dalloc_t(c, dst, count > 0 ? count : 1));
    if (count) CPTR_CUDA_TRY(c, cudaMemcpyAsync(*dst, src, sizeof(I) * count, cudaMemcpyDeviceToDevice, c->stream));
    return CPTR_OK;
}

static void pair_free(Ctx *c) {
    void **sp[] = {(void **)&c->sp_off_f, (void **)&c->sp_off_b, (void **)&c->sp_coff_f, (void **)&c->sp_coff_b,
                   (void **)&c->sp_col_f, (void **)&c->sp_col_b, (void **)&c->sp_ccol_f, (void **)&c->sp_ccol_b,
                   (void **)&c->sp_val_f, (void **)&c->sp_val_b, (void **)&c->sp_cval_f, (void **)&c->sp_cval_b};
    for (void **p : sp) { dfree(*p); *p = nullptr; }
    c->sp_ok = false;
    c->sp_group = 0;
}

// the grouped-level tables of one sweep (G levels per group); *ok = false when an expanded row has
// too many entries
static cptr_status pair_table(Ctx *c, bool lower, int G, const int32_t *pos, const int32_t *inv, const int32_t *levr,
                              const int32_t *src_of_row, int64_t **off, int32_t **col, void **val, int64_t **coff,
                              int32_t **ccol, void **cval, bool *ok) {
    const int32_t n = c->n, nch = (n + 31) / 32, BB = c->b * c->b;
    cudaStream_t s = c->stream;
    // the structure of a set-up of the same pattern with the same group size, if kept
    IluSym &ys = c->isym;
    IluSym::GroupDir *gd = ys.current ? &ys.gd[lower ? 0 : 1] : nullptr;
    const bool cached = gd && ys.grp == G && gd->mcnt;
    int32_t *mcnt = nullptr, *ccnt = nullptr, *moff = nullptr, *coffc = nullptr, *mdep = nullptr, *cdep = nullptr;
    int32_t mtot = 0, ctot = 0;
    if (cached) {
        mcnt = gd->mcnt; ccnt = gd->ccnt; moff = gd->moff; coffc = gd->coff; mdep = gd->mdep; cdep = gd->cdep;
        mtot = gd->mtot;
        ctot = gd->ctot;
        *ok = true;
    } else {
        int32_t *err = nullptr;
        CPTR_TRY(dalloc_t(c, &mcnt, (size_t)n + 1));
        CPTR_TRY(dalloc_t(c, &ccnt, (size_t)n + 1));
        CPTR_TRY(dalloc_t(c, &moff, (size_t)n + 1));
        CPTR_TRY(dalloc_t(c, &coffc, (size_t)n + 1));
        CPTR_TRY(dalloc_t(c, &err, 1));
        CPTR_CUDA_TRY(c, cudaMemsetAsync(err, 0, sizeof(int32_t), s));
        (k_group_count<<<nblk(n, 128), 128, 0, s>>>(n, pos, inv, c->ilu_rp, c->ilu_ci, c->ilu_diag, levr, lower ? 1 : 0,
                                                    G, src_of_row, mcnt, ccnt, err),
         note_launch());
        CPTR_TRY(scan_exclusive(c, mcnt, moff, n, nullptr));
        CPTR_TRY(scan_exclusive(c, ccnt, coffc, n, nullptr));
        int32_t rd[3] = {0, 0, 0};   // both totals and the overflow flag, one synchronisation
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(&rd[0], moff + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(&rd[1], coffc + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(&rd[2], err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CPTR_CUDA_TRY(c, cudaStreamSynchronize(s));
        dfree(err);
        mtot = rd[0];
        ctot = rd[1];
        *ok = !rd[2];
        if (*ok) {
            CPTR_TRY(dalloc_t(c, &mdep, (size_t)(mtot > 0 ? mtot : 1)));
            CPTR_TRY(dalloc_t(c, &cdep, (size_t)(ctot > 0 ? ctot : 1)));
        }
    }
    if (*ok) {
        double *mblk = nullptr, *cblk = nullptr;
        CPTR_TRY(dalloc_t(c, &mblk, (size_t)(mtot > 0 ? mtot : 1) * BB));
        CPTR_TRY(dalloc_t(c, &cblk, (size_t)(ctot > 0 ? ctot : 1) * BB));
        for (int p = 0; p < G; ++p) {   // one pass per position in the group: earlier positions first
            auto fill = [&](auto kern) {
                (kern<<<nblk(n, 128), 128, 0, s>>>(n, pos, inv, c->ilu_rp, c->ilu_ci, c->ilu_diag, levr, lower ? 1 : 0,
                                                   G, p, c->LU, src_of_row, mcnt, ccnt, moff, coffc, mdep, mblk, cdep,
                                                   cblk),
                 note_launch());
            };
            if (c->b == 3) fill(k_group_fill<3>);
            else fill(k_group_fill<4>);
        }
        if (!lower) {   // the backward blocks with the rows' inverted pivots folded in
            if (c->b == 3)
                (k_group_fold<3><<<nblk(n, 128), 128, 0, s>>>(n, pos, c->ilu_diag, c->LU, mcnt, ccnt, moff, coffc, mblk,
                                                             cblk), note_launch());
            else
                (k_group_fold<4><<<nblk(n, 128), 128, 0, s>>>(n, pos, c->ilu_diag, c->LU, mcnt, ccnt, moff, coffc, mblk,
                                                             cblk), note_launch());
        }
        if (cached) {   // the kept SELL layouts, values packed anew
            CPTR_TRY(dcopy(c, off, gd->off[0], (size_t)nch + 1));
            CPTR_TRY(dcopy(c, col, gd->col[0], (size_t)gd->ns[0]));
            CPTR_TRY(dcopy(c, coff, gd->off[1], (size_t)nch + 1));
            CPTR_TRY(dcopy(c, ccol, gd->col[1], (size_t)gd->ns[1]));
            CPTR_TRY(sell_pack(c, gd->kidx[0], gd->ns[0], mblk, val));
            CPTR_TRY(sell_pack(c, gd->kidx[1], gd->ns[1], cblk, cval));
        } else {
            int32_t *kidx[2] = {};
            int64_t ns[2] = {};
            CPTR_TRY(sell_layout(c, mcnt, moff, mdep, off, col, &kidx[0], &ns[0]));
            CPTR_TRY(sell_layout(c, ccnt, coffc, cdep, coff, ccol, &kidx[1], &ns[1]));
            CPTR_TRY(sell_pack(c, kidx[0], ns[0], mblk, val));
            CPTR_TRY(sell_pack(c, kidx[1], ns[1], cblk, cval));
            if (gd) {   // kept for the next set-up of this pattern (group size recorded by the caller)
                IluSym::GroupDir &g = *gd;
                dfree(g.mcnt); dfree(g.ccnt); dfree(g.moff); dfree(g.coff); dfree(g.mdep); dfree(g.cdep);
                for (int t = 0; t < 2; ++t) { dfree(g.off[t]); dfree(g.col[t]); dfree(g.kidx[t]); }
                g = IluSym::GroupDir();
                g.mcnt = mcnt; g.ccnt = ccnt; g.moff = moff; g.coff = coffc; g.mdep = mdep; g.cdep = cdep;
                g.mtot = mtot;
                g.ctot = ctot;
                CPTR_TRY(dcopy(c, &g.off[0], *off, (size_t)nch + 1));
                CPTR_TRY(dcopy(c, &g.col[0], *col, (size_t)ns[0]));
                CPTR_TRY(dcopy(c, &g.off[1], *coff, (size_t)nch + 1));
                CPTR_TRY(dcopy(c, &g.col[1], *ccol, (size_t)ns[1]));
                g.kidx[0] = kidx[0];
                g.kidx[1] = kidx[1];
                g.ns[0] = ns[0];
                g.ns[1] = ns[1];
                mcnt = ccnt = moff = coffc = mdep = cdep = nullptr;   // owned by the cache now
            } else {
                dfree(kidx[0]); dfree(kidx[1]);
            }
        }
        dfree(mblk); dfree(cblk);   // (stream-ordered frees)
    }
    if (!cached) { dfree(mcnt); dfree(ccnt); dfree(moff); dfree(coffc); dfree(mdep); dfree(cdep); }
    return CPTR_OK;
}

// both sweeps' grouped-level tables with G levels per group (blocks in the sweeps' precision);
// c->sp_ok tells whether they were built, c->sp_group their group size.  Tables built before are
// dropped first.
static cptr_status pair_setup(Ctx *c, int G) {
    pair_free(c);
    // a kept structure of another group size is replaced direction by direction below: until both
    // are built it belongs to no group size
    if (c->isym.grp != G) c->isym.grp = 0;
    bool okf = false, okb = false;
    CPTR_TRY(pair_table(c, true, G, c->lvl_f, c->sp_inv_f, c->sp_levr_f, c->ilu_rowmap, &c->sp_off_f, &c->sp_col_f,
                        &c->sp_val_f, &c->sp_coff_f, &c->sp_ccol_f, &c->sp_cval_f, &okf));
    if (okf)
        CPTR_TRY(pair_table(c, false, G, c->lvl_b, c->sp_inv_b, c->sp_levr_b, c->sp_inv_f, &c->sp_off_b, &c->sp_col_b,
                            &c->sp_val_b, &c->sp_coff_b, &c->sp_ccol_b, &c->sp_cval_b, &okb));
    c->sp_ok = okf && okb;
    c->sp_group = c->sp_ok ? G : 0;
    if (c->isym.current) c->isym.grp = c->sp_ok ? G : 0;   // the kept structure's group size (both sweeps)
    if (!c->sp_ok) pair_free(c);
    return CPTR_OK;
}

// key of the sweeps' tuning in the context's cache (grid and back-off; the schedule at key + 1)
static uint64_t ilu_tune_key(const Ctx *c) {
    return (uint64_t)8 << 60 | (uint64_t)(c->part != nullptr) << 58 | (uint64_t)(c->o.ilu_fill & 1) << 57 |
           (uint64_t)(c->o.precision & 1) << 56 |
           ((uint64_t)c->n & 0xFFFFFFull) << 32 |
           (uint64_t)(uint32_t)c->nnzb;
}
// the schedule a cached tuning chose (0 level sets, 1 chunked, 2 paired levels, 3 tiled), -1 if
// none; the tiled schedule's tile shape is cached at key + 2 (G = Ty, T = Tz)
static int ilu_tuned_schedule(const Ctx *c) {
    auto it = c->tune_cache.find(ilu_tune_key(c) + 1);
    return it == c->tune_cache.end() ? -1 : it->second.G;
}
// levels per group of the grouped-level tables: the caller's, else the one a cached tuning chose
// (kept at key + 1 as T), else two
static int ilu_group_size(const Ctx *c) {
    if (c->o.ilu_group >= 2) return c->o.ilu_group;
    auto it = c->tune_cache.find(ilu_tune_key(c) + 1);
    if (it != c->tune_cache.end() && it->second.G == 2 && it->second.T >= 2) return it->second.T;
    return 2;
}

// Block ILU(1) pattern (Sec. 4; the CPR-AMG-ILU(1) comparator): block row i keeps its own blocks and
// gains, for every block k < i of its row, the blocks j > k of row k -- a fill block has level
// lev(i,k) + lev(k,j) + 1, at most 1 only when both are original blocks.  kmap: the original block of
// every position of the new pattern, -1 at fill.  Rows are built on up to 8 host threads.
static void ilu1_pattern(int32_t n, const std::vector<int32_t> &rp, const std::vector<int32_t> &ci,
                         std::vector<int32_t> &prp, std::vector<int32_t> &pci, std::vector<int32_t> &pdg,
                         std::vector<int32_t> &kmap) {
    std::vector<std::vector<int32_t>> rows(n);
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nt = (int)std::min<unsigned>(8u, hw);
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t)
        pool.emplace_back([&, t]() {
            std::vector<int32_t> cols;
            for (int32_t i = t; i < n; i += nt) {
                cols.assign(ci.begin() + rp[i], ci.begin() + rp[i + 1]);
                for (int32_t k = rp[i]; k < rp[i + 1] && ci[k] < i; ++k) {
                    const int32_t kc = ci[k];
                    for (int32_t q = rp[kc]; q < rp[kc + 1]; ++q)
                        if (ci[q] > kc) cols.push_back(ci[q]);
                }
                std::sort(cols.begin(), cols.end());
                cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
                rows[i] = cols;
            }
        });
    for (auto &th : pool) th.join();
    prp.assign((size_t)n + 1, 0);
    for (int32_t i = 0; i < n; ++i) prp[i + 1] = prp[i] + (int32_t)rows[i].size();
    pci.resize(prp[n]);
    kmap.assign(prp[n], -1);
    pdg.assign(n, -1);
    for (int32_t i = 0; i < n; ++i) {
        int32_t a = rp[i];
        for (size_t t = 0; t < rows[i].size(); ++t) {
            const int32_t o = prp[i] + (int32_t)t, j = rows[i][t];
            pci[o] = j;
            if (a < rp[i + 1] && ci[a] == j) kmap[o] = a++;
            if (j == i) pdg[i] = o;
        }
    }
}

__global__ void k_scatter_blocks(int64_t nnz, int BB, const int32_t *kmap, const double *src, double *dst) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nnz * BB) return;
    const int32_t k = kmap[u / BB];
    dst[u] = k >= 0 ? src[(int64_t)k * BB + u % BB] : 0.0;
}

// Block-Jacobi pattern (Sec. 4: in parallel, ILU(k) is applied to each block of the domain's
// partition): row i keeps the blocks whose column lies in its own part.  kmap: the original block
// of every kept position; pdg: the kept diagonal's position.
__global__ void k_part_count(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                             const int32_t *__restrict__ part, int32_t *cnt) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t pi = part[i];
    int32_t c = 0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) c += part[ci[k]] == pi;
    cnt[i] = c;
}
__global__ void k_part_fill(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const int32_t *__restrict__ part, const int32_t *__restrict__ prp, int32_t *pci,
                            int32_t *pdg, int32_t *kmap) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t pi = part[i];
    int32_t o = prp[i];
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
        const int32_t j = ci[k];
        if (part[j] != pi) continue;
        if (j == i) pdg[i] = o;
        pci[o] = j;
        kmap[o] = k;
        ++o;
    }
}

// 1 in *diff if the pattern (rp, ci) differs from (srp, sci) anywhere
__global__ void k_pattern_diff(int32_t n, int32_t nnzb, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                               const int32_t *__restrict__ srp, const int32_t *__restrict__ sci, int32_t *diff) {
    bool d = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnzb; i += (int64_t)gridDim.x * blockDim.x) {
        if (ci[i] != sci[i]) d = true;
        if (i <= n && rp[i] != srp[i]) d = true;
    }
    if (__syncthreads_or(d) && threadIdx.x == 0) *diff = 1;
}

void ilu_sym_free(Ctx *c) {
    IluSym &y = c->isym;
    dfree(y.rp); dfree(y.ci);
    for (int d = 0; d < 2; ++d) {
        dfree(y.lvl[d]); dfree(y.inv[d]); dfree(y.levr[d]);
        dfree(y.tt[d].tlev); dfree(y.tt[d].lptr); dfree(y.hdr[d]); dfree(y.kidx[d]);
        IluSym::GroupDir &g = y.gd[d];
        dfree(g.mcnt); dfree(g.ccnt); dfree(g.moff); dfree(g.coff); dfree(g.mdep); dfree(g.cdep);
        for (int t = 0; t < 2; ++t) { dfree(g.off[t]); dfree(g.col[t]); dfree(g.kidx[t]); }
    }
    y = IluSym();
}

// Whether the tables of c->isym belong to this set-up's pattern and ILU options; if not, they are
// dropped and the pattern is recorded for the tables this set-up builds.
static cptr_status ilu_sym_check(Ctx *c, bool *same) {
    IluSym &y = c->isym;
    *same = false;
    const int32_t n = c->n, nnzb = c->nnzb;
    if (y.rp && y.n == n && y.b == c->b && y.nnzb == nnzb && y.order == c->o.ilu_order && y.fill == c->o.ilu_fill) {
        int32_t *diff = c->flag + 2, h = 1;
        CPTR_CUDA_TRY(c, cudaMemsetAsync(diff, 0, sizeof(int32_t), c->stream));
        (k_pattern_diff<<<std::min<unsigned>(nblk(nnzb, 256), 4 * 152), 256, 0, c->stream>>>(n, nnzb, c->rp, c->ci, y.rp,
                                                                                              y.ci, diff), note_launch());
        CPTR_TRY(copy_to_host(c, &h, diff, sizeof(int32_t)));
        *same = h == 0;
    }
    if (!*same) {
        ilu_sym_free(c);
        CPTR_TRY(dalloc_t(c, &y.rp, (size_t)n + 1));
        CPTR_TRY(dalloc_t(c, &y.ci, (size_t)nnzb));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(y.rp, c->rp, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToDevice, c->stream));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(y.ci, c->ci, sizeof(int32_t) * (size_t)nnzb, cudaMemcpyDeviceToDevice, c->stream));
        y.n = n;
        y.b = c->b;
        y.nnzb = nnzb;
        y.order = c->o.ilu_order;
        y.fill = c->o.ilu_fill;
    }
    y.current = true;
    return CPTR_OK;
}

static cptr_status d2d_copy(Ctx *c, int32_t *dst, const int32_t *src, size_t count) {
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(dst, src, sizeof(int32_t) * count, cudaMemcpyDeviceToDevice, c->stream));
    return CPTR_OK;
}

cptr_status ilu_setup(Ctx *c) {
    ilu_free(c);
    double t0 = host_ms();
    bool same_pattern = false;
    CPTR_TRY(ilu_sym_check(c, &same_pattern));
    const int32_t n = c->n, BB = c->b * c->b;
    cudaStream_t st = c->stream;
    // the pattern the factorisation works on: the caller's order, cells permuted by colour, the
    // ILU(1) fill pattern, or the caller's pattern without the couplings between parts (block Jacobi)
    std::vector<int32_t> rowmap;
    const bool mc = c->o.ilu_order == CPTR_ILU_MULTICOLOR;
    const bool fill = c->o.ilu_fill == 1;
    const bool bj = c->part != nullptr;
    if (bj && (c->n_part != n || mc || fill))
        return c->fail(CPTR_EINVAL, c->n_part != n ? "the partition's cell count differs from the set-up's"
                                                   : "the block-Jacobi ILU(0) needs the natural order and no fill");
    int64_t nnz_ilu = c->nnzb;
    if (bj) {
        int32_t *cnt = nullptr, *dk = nullptr;
        CPTR_TRY(dalloc_t(c, &cnt, (size_t)n + 1));
        CPTR_TRY(dalloc_t(c, &c->ilu_rp, (size_t)n + 1));
        c->ilu_owns_pattern = true;
        (k_part_count<<<nblk(n, 256), 256, 0, st>>>(n, c->rp, c->ci, c->part, cnt), note_launch());
        int32_t total = 0;
        CPTR_TRY(scan_exclusive(c, cnt, c->ilu_rp, n, &total));
        nnz_ilu = total;
        CPTR_TRY(dalloc_t(c, &c->ilu_ci, (size_t)nnz_ilu));
        CPTR_TRY(dalloc_t(c, &c->ilu_diag, (size_t)n));
        CPTR_TRY(dalloc_t(c, &dk, (size_t)nnz_ilu));
        (k_part_fill<<<nblk(n, 256), 256, 0, st>>>(n, c->rp, c->ci, c->part, c->ilu_rp, c->ilu_ci, c->ilu_diag, dk),
         note_launch());
        // two spare doubles: the factorisation copies runs of blocks in 16-byte pieces rounded outwards
        CPTR_TRY(dalloc_t(c, &c->LU, (size_t)nnz_ilu * BB + 2));
        (k_scatter_blocks<<<nblk(nnz_ilu * BB, 256), 256, 0, st>>>(nnz_ilu, BB, dk, c->A, c->LU), note_launch());
        CPTR_CUDA_TRY(c, cudaStreamSynchronize(st));
        dfree(cnt);
        dfree(dk);
    } else if (fill) {
        CPTR_TRY(host_pattern(c));
        std::vector<int32_t> prp, pci, pdg, kmap;
        ilu1_pattern(n, c->h_rp, c->h_ci, prp, pci, pdg, kmap);
        nnz_ilu = prp[n];
        c->ilu_owns_pattern = true;
        CPTR_TRY(dalloc_t(c, &c->ilu_rp, (size_t)n + 1));
        CPTR_TRY(dalloc_t(c, &c->ilu_ci, (size_t)nnz_ilu));
        CPTR_TRY(dalloc_t(c, &c->ilu_diag, (size_t)n));
        // two spare doubles: the factorisation copies runs of blocks in 16-byte pieces rounded outwards
        CPTR_TRY(dalloc_t(c, &c->LU, (size_t)nnz_ilu * BB + 2));
        int32_t *dk = nullptr;
        CPTR_TRY(dalloc_t(c, &dk, (size_t)nnz_ilu));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->ilu_rp, prp.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, st));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->ilu_ci, pci.data(), sizeof(int32_t) * nnz_ilu, cudaMemcpyHostToDevice, st));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->ilu_diag, pdg.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(dk, kmap.data(), sizeof(int32_t) * nnz_ilu, cudaMemcpyHostToDevice, st));
        (k_scatter_blocks<<<nblk(nnz_ilu * BB, 256), 256, 0, st>>>(nnz_ilu, BB, dk, c->A, c->LU), note_launch());
        CPTR_CUDA_TRY(c, cudaStreamSynchronize(st));
        dfree(dk);
    } else {
        // two spare doubles: the factorisation copies runs of blocks in 16-byte pieces rounded outwards
        CPTR_TRY(dalloc_t(c, &c->LU, (size_t)c->nnzb * BB + 2));
    }
    if (fill || bj) {
    } else if (mc) {
        CPTR_TRY(host_pattern(c));
        rowmap = multicolour_order(n, c->h_rp, c->h_ci);
        std::vector<int32_t> inv(n), kmap(c->nnzb), prp(n + 1, 0), pci(c->nnzb), pdg(n, -1);
        for (int32_t I = 0; I < n; ++I) inv[rowmap[I]] = I;
        std::vector<std::pair<int32_t, int32_t>> row;
        for (int32_t I = 0; I < n; ++I) {
            int32_t i = rowmap[I];
            row.clear();
            for (int32_t k = c->h_rp[i]; k < c->h_rp[i + 1]; ++k) row.push_back({inv[c->h_ci[k]], k});
            std::sort(row.begin(), row.end());
            int32_t o = prp[I];
            for (auto &pr : row) {
                pci[o] = pr.first;
                kmap[o] = pr.second;
                if (pr.first == I) pdg[I] = o;
                ++o;
            }
            prp[I + 1] = o;
        }
        c->ilu_owns_pattern = true;
        CPTR_TRY(dalloc_t(c, &c->ilu_rp, (size_t)n + 1));
        CPTR_TRY(dalloc_t(c, &c->ilu_ci, (size_t)c->nnzb));
        CPTR_TRY(dalloc_t(c, &c->ilu_diag, (size_t)n));
        CPTR_TRY(dalloc_t(c, &c->ilu_rowmap, (size_t)n));
        int32_t *dk = nullptr;
        CPTR_TRY(dalloc_t(c, &dk, (size_t)c->nnzb));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->ilu_rp, prp.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, st));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->ilu_ci, pci.data(), sizeof(int32_t) * c->nnzb, cudaMemcpyHostToDevice, st));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->ilu_diag, pdg.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->ilu_rowmap, rowmap.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(dk, kmap.data(), sizeof(int32_t) * c->nnzb, cudaMemcpyHostToDevice, st));
        (k_gather_blocks<<<nblk((int64_t)c->nnzb * BB, 256), 256, 0, st>>>(c->nnzb, BB, dk, c->A, c->LU), note_launch());
        CPTR_CUDA_TRY(c, cudaStreamSynchronize(st));
        dfree(dk);
    } else {
        c->ilu_rp = c->rp;
        c->ilu_ci = c->ci;
        c->ilu_diag = c->diag;
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->LU, c->A, sizeof(double) * (size_t)c->nnzb * BB, cudaMemcpyDeviceToDevice, st));
    }
    // level sets of both sweeps (positions -> rows of the factorised matrix)
    // (positions and levels stay with the context: the autotuner rebuilds grouped-level tables)
    CPTR_TRY(dalloc_t(c, &c->lvl_f, (size_t)n));
    CPTR_TRY(dalloc_t(c, &c->lvl_b, (size_t)n));
    CPTR_TRY(dalloc_t(c, &c->sp_inv_f, (size_t)n));
    CPTR_TRY(dalloc_t(c, &c->sp_inv_b, (size_t)n));
    CPTR_TRY(dalloc_t(c, &c->sp_levr_f, (size_t)n));
    CPTR_TRY(dalloc_t(c, &c->sp_levr_b, (size_t)n));
    int32_t *inv_f = c->sp_inv_f, *inv_b = c->sp_inv_b, *levr_f = c->sp_levr_f, *levr_b = c->sp_levr_b;
    IluSym &ys = c->isym;
    if (ys.lv) {   // the level sets of the same pattern, from the last set-up
        int32_t *dst[6] = {c->lvl_f, inv_f, levr_f, c->lvl_b, inv_b, levr_b};
        const int32_t *src[6] = {ys.lvl[0], ys.inv[0], ys.levr[0], ys.lvl[1], ys.inv[1], ys.levr[1]};
        for (int q = 0; q < 6; ++q) CPTR_TRY(d2d_copy(c, dst[q], src[q], (size_t)n));
        c->h_lptr_f = ys.lptr[0];
        c->h_lptr_b = ys.lptr[1];
    } else {
        CPTR_TRY(device_levels(c, c->ilu_rp, c->ilu_ci, c->lvl_f, inv_f, c->h_lptr_f, c->lvl_b, inv_b, c->h_lptr_b,
                               levr_f, levr_b));
        const int32_t *src[6] = {c->lvl_f, inv_f, levr_f, c->lvl_b, inv_b, levr_b};
        int32_t **dst[6] = {&ys.lvl[0], &ys.inv[0], &ys.levr[0], &ys.lvl[1], &ys.inv[1], &ys.levr[1]};
        for (int q = 0; q < 6; ++q) {
            CPTR_TRY(dalloc_t(c, dst[q], (size_t)n));
            CPTR_TRY(d2d_copy(c, *dst[q], src[q], (size_t)n));
        }
        ys.lptr[0] = c->h_lptr_f;
        ys.lptr[1] = c->h_lptr_b;
        ys.lv = true;
    }
    c->nlev_f = (int32_t)c->h_lptr_f.size() - 1;
    c->nlev_b = (int32_t)c->h_lptr_b.size() - 1;
    CPTR_TRY(dalloc_t(c, &c->ybuf, (size_t)n * c->b));
    CPTR_TRY(dalloc_t(c, &c->zbuf, (size_t)n * c->b));
    setup_tick(c, SETUP_ILU_HOST, &t0);
    // factorisation, one launch
    CPTR_TRY(dalloc_t(c, &c->sf_ticket, 4));
    if (c->ilu_flags && c->ilu_flags_n != n) {
        dfree(c->ilu_flags);
        c->ilu_flags = nullptr;
    }
    if (!c->ilu_flags) {
        CPTR_TRY(dalloc_t(c, &c->ilu_flags, (size_t)n));
        CPTR_CUDA_TRY(c, cudaMemsetAsync(c->ilu_flags, 0, sizeof(int32_t) * n, st));
        c->ilu_flags_n = n;
        c->ilu_epoch = 0;
    }
    ++c->ilu_epoch;
    int32_t *fsing = c->flag + 3;   // the factorisation's singular flag
    CPTR_CUDA_TRY(c, cudaMemsetAsync(fsing, 0, sizeof(int32_t), st));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(c->sf_ticket, 0, 4 * sizeof(unsigned), st));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(reinterpret_cast<char *>(c->ks) + offsetof(KState, wait_err), 0, sizeof(int32_t), st));
    // per-row sizes of the pattern: the factorisation kernel holds a row, and the pivot inverse and upper
    // blocks of each dependency, in shared memory when that fits
    int maxrow = 0, maxdep = 0, maxu = 0;
    {
        int32_t *ext = nullptr, h_ext[3] = {0, 0, 0};
        CPTR_TRY(dalloc_t(c, &ext, 3));
        CPTR_CUDA_TRY(c, cudaMemsetAsync(ext, 0, 3 * sizeof(int32_t), st));
        (k_row_extents<<<nblk(n, 256), 256, 0, st>>>(n, c->ilu_rp, c->ilu_ci, ext), note_launch());
        const cptr_status cs = copy_to_host(c, h_ext, ext, sizeof(h_ext));
        dfree(ext);
        CPTR_TRY(cs);
        maxrow = h_ext[0];
        maxdep = h_ext[1];
        maxu = h_ext[2];
    }
    const unsigned fgrid = std::min<unsigned>(nblk(n, 64), 8 * 152);
    // a row per warp (k_bilu_factor_w) while its tables fit; one row per thread otherwise
    const size_t fw_bytes = (size_t)kFwWarps * ((size_t)fw_warp_doubles(c->b, maxrow, maxdep, maxu) * 8 +
                                                 (size_t)fw_warp_ints(maxrow, maxdep, maxu) * 4);
    const size_t fs_rowsz = (size_t)((maxrow * BB + 1) & ~1), fs_w = (size_t)(((1 + maxu) * BB + 3) & ~1);
    const size_t fg_bytes = (size_t)kSfRowsG * ((fs_rowsz + (size_t)maxdep * fs_w) * 8 +
                                                (size_t)(maxrow + maxdep * (2 + maxu)) * 4);
    // Narrow levels (up to ~2000 rows on average) are latency bound: a row per warp issues the
    // fewest FP64 instructions per row's chain.  Wide levels are bound by the FP64 pipe's
    // throughput, where a row over four lanes issues ~2.5x fewer FP64 instructions per row.
    const bool narrow = (double)n <= 2000.0 * std::max<int32_t>(c->nlev_f, 1);
    if (narrow && fw_bytes <= 100 * 1024) {
        // two blocks per SM: rows a few levels ahead of the wavefront are taken and wait on their
        // flags, so a level's rows start as soon as the last of their dependencies is published
        const unsigned wgrid = std::min<unsigned>(nblk(n, kFwWarps), 2 * 152);
        if (c->b == 3) {
            cudaFuncSetAttribute(k_bilu_factor_w<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
            (k_bilu_factor_w<3><<<wgrid, 32 * kFwWarps, fw_bytes, st>>>(n, c->sf_ticket, c->lvl_f, c->ilu_rp, c->ilu_ci,
                                                                         c->ilu_diag, c->LU, c->ilu_flags, c->ilu_epoch,
                                                                         fsing, c->ks, maxrow, maxdep, maxu),
             note_launch());
        } else {
            cudaFuncSetAttribute(k_bilu_factor_w<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
            (k_bilu_factor_w<4><<<wgrid, 32 * kFwWarps, fw_bytes, st>>>(n, c->sf_ticket, c->lvl_f, c->ilu_rp, c->ilu_ci,
                                                                         c->ilu_diag, c->LU, c->ilu_flags, c->ilu_epoch,
                                                                         fsing, c->ks, maxrow, maxdep, maxu),
             note_launch());
        }
    } else if (fg_bytes <= 100 * 1024) {
        // one block per SM (32 rows each, a few levels ahead of the wavefront): more rows in flight
        // only poll, and measured slower.  Two SMs are left to the coarsest AMG inverses.
        const unsigned ggrid = std::min<unsigned>(nblk(n, kSfRowsG), 150u);
        if (c->b == 3) {
            cudaFuncSetAttribute(k_bilu_factor_g<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
            (k_bilu_factor_g<3><<<ggrid, kSfThreads, fg_bytes, st>>>(n, c->sf_ticket, c->lvl_f, c->ilu_rp, c->ilu_ci,
                                                                      c->ilu_diag, c->LU, c->ilu_flags, c->ilu_epoch,
                                                                      fsing, c->ks, maxrow, maxdep, maxu), note_launch());
        } else {
            cudaFuncSetAttribute(k_bilu_factor_g<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
            (k_bilu_factor_g<4><<<ggrid, kSfThreads, fg_bytes, st>>>(n, c->sf_ticket, c->lvl_f, c->ilu_rp, c->ilu_ci,
                                                                      c->ilu_diag, c->LU, c->ilu_flags, c->ilu_epoch,
                                                                      fsing, c->ks, maxrow, maxdep, maxu), note_launch());
        }
    } else if (c->b == 3)
        (k_bilu_factor_sf<3><<<fgrid, 64, 0, st>>>(n, c->sf_ticket, c->lvl_f, c->ilu_rp, c->ilu_ci, c->ilu_diag, c->LU,
                                                    c->ilu_flags, c->ilu_epoch, fsing, c->ks), note_launch());
    else
        (k_bilu_factor_sf<4><<<fgrid, 64, 0, st>>>(n, c->sf_ticket, c->lvl_f, c->ilu_rp, c->ilu_ci, c->ilu_diag, c->LU,
                                                    c->ilu_flags, c->ilu_epoch, fsing, c->ks), note_launch());
    CPTR_CUDA_TRY(c, cudaGetLastError());
    int32_t sing = 0, werr = 0;
    CPTR_TRY(copy_to_host(c, &sing, fsing, sizeof(int32_t)));
    CPTR_TRY(copy_to_host(c, &werr, reinterpret_cast<char *>(c->ks) + offsetof(KState, wait_err), sizeof(int32_t)));
    if (werr) return c->fail(CPTR_ETIMEOUT, "ILU(0) factorisation: a bounded wait gave up");
    if (sing) return c->fail(CPTR_ESINGULAR, "ILU(0): singular pivot block");
    setup_tick(c, SETUP_ILU_FACTOR, &t0);
    // sweep tables: positions of the sweeps in the caller's row order, dependency tables, factors
    const int32_t nch = (n + 31) / 32;
    CPTR_TRY(dalloc_t(c, &c->sf_pos_f, (size_t)n));
    CPTR_TRY(dalloc_t(c, &c->sf_pos_b, (size_t)n));
    CPTR_TRY(dalloc_t(c, &c->sf_bmap, (size_t)n));
    if (mc) {
        (k_compose<<<nblk(n, 256), 256, 0, st>>>(n, c->ilu_rowmap, c->lvl_f, c->sf_pos_f), note_launch());
        (k_compose<<<nblk(n, 256), 256, 0, st>>>(n, c->ilu_rowmap, c->lvl_b, c->sf_pos_b), note_launch());
    } else {
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->sf_pos_f, c->lvl_f, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->sf_pos_b, c->lvl_b, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st));
    }
    (k_compose<<<nblk(n, 256), 256, 0, st>>>(n, inv_f, c->lvl_b, c->sf_bmap), note_launch());
    const bool lo = c->o.precision == CPTR_PREC_MIXED;   // factors stored in FP32
    // paired-level tables first: when they are the schedule in use (forced, or chosen by a cached
    // tuning), the level-set tables of L and U are not needed
    const int sched = ilu_tuned_schedule(c);
    if (c->o.ilu_sweep == 3 || (c->o.ilu_sweep == 0 && c->o.autotune && (sched < 0 || sched == 2))) {
        CPTR_TRY(pair_setup(c, ilu_group_size(c)));
        c->sp_use = c->sp_ok && (c->o.ilu_sweep == 3 || sched == 2);
        c->sf_half = c->o.ilu_lanes ? c->o.ilu_lanes / 4 : 1;   // (a cached tuning's choice is restored by the autotuner)
    }
    int32_t *kidx_f = nullptr, *kidx_b = nullptr, *kidx_d = nullptr;
    int64_t ns_f = 0, ns_b = 0;
    auto pack = [&](const int32_t *kidx, int64_t ns, void **dst) -> cptr_status {
        CPTR_TRY(dalloc(c, dst, (size_t)(ns > 0 ? ns : 1) * BB * (lo ? 4 : 8)));
        if (ns == 0) return CPTR_OK;
        if (lo) (k_sf_pack<float><<<nblk(ns, 256), 256, 0, st>>>(ns, BB, kidx, c->LU, (float *)*dst), note_launch());
        else (k_sf_pack<double><<<nblk(ns, 256), 256, 0, st>>>(ns, BB, kidx, c->LU, (double *)*dst), note_launch());
        return CPTR_OK;
    };
    if (!c->sp_use) {
        CPTR_TRY(device_table(c, c->lvl_f, inv_f, c->ilu_rp, c->ilu_ci, c->ilu_diag, true, &c->sf_off_f, &c->sf_col_f,
                              &kidx_f, &ns_f));
        CPTR_TRY(device_table(c, c->lvl_b, inv_b, c->ilu_rp, c->ilu_ci, c->ilu_diag, false, &c->sf_off_b,
                              &c->sf_col_b, &kidx_b, &ns_b));
        CPTR_TRY(pack(kidx_f, ns_f, &c->sf_val_f));
        CPTR_TRY(pack(kidx_b, ns_b, &c->sf_val_b));
    }
    CPTR_TRY(dalloc_t(c, &kidx_d, (size_t)nch * 32));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(kidx_d, 0xFF, sizeof(int32_t) * nch * 32, st));
    (k_dinv_index<<<nblk(n, 256), 256, 0, st>>>(n, c->lvl_b, c->ilu_diag, kidx_d), note_launch());
    CPTR_TRY(pack(kidx_d, (int64_t)nch * 32, &c->sf_dinv));
    // (+64 bytes: the chunked sweeps read 32-byte windows around a row's values)
    CPTR_TRY(dalloc(c, &c->sf_y, (size_t)n * c->b * (lo ? 4 : 8) + 64));
    CPTR_TRY(dalloc(c, &c->sf_z, (size_t)n * c->b * (lo ? 4 : 8) + 64));
    CPTR_CUDA_TRY(c, cudaGetLastError());
    dfree(kidx_f); dfree(kidx_b); dfree(kidx_d);
    // the chunked and tiled schedules read the caller's pattern: natural order without fill only
    if (!mc && !fill && !bj && (c->o.ilu_sweep == 2 || (c->o.ilu_sweep == 0 && c->o.autotune && (sched < 0 || sched == 1))))
        CPTR_TRY(cw_setup(c));
    // tiled sweeps: on a natural-order box, with the cached tile shape or the best modelled one
    c->tl_use = false;
    if (!mc && !fill && !bj && (c->o.ilu_sweep == 4 || (c->o.ilu_sweep == 0 && c->o.autotune && (sched < 0 || sched == 3))) &&
        tile_grid(c)) {
        int Ty = 0, Tz = 0;
        auto it = c->tune_cache.find(ilu_tune_key(c) + 2);
        if (c->o.tile_y > 0 || c->o.tile_z > 0) {   // the caller's shape (clamped to the box)
            Ty = std::min(std::max(c->o.tile_y, 1), c->tl_dims[1]);
            Tz = std::min(std::max(c->o.tile_z, 1), c->tl_dims[2]);
        } else if (it != c->tune_cache.end()) {
            Ty = it->second.G;
            Tz = it->second.T;
        } else {
            std::vector<std::pair<int, int>> cand;
            tile_candidates(c, 1, cand);
            if (!cand.empty()) { Ty = cand[0].first; Tz = cand[0].second; }
        }
        if (Ty > 0) CPTR_TRY(tile_setup(c, Ty, Tz));
        c->tl_use = c->tl_ok && (c->o.ilu_sweep == 4 || sched == 3);
        if (c->tl_ok) { c->tl_best_ty = c->tl_ty; c->tl_best_tz = c->tl_tz; }
    }
    setup_tick(c, SETUP_ILU_HOST, &t0);
    return CPTR_OK;
}

void ilu_free(Ctx *c) {
    cw_free(c);
    tile_free(c);
    c->tl_use = false;
    c->isym.current = false;
    if (c->ilu_owns_pattern) { dfree(c->ilu_rp); dfree(c->ilu_ci); dfree(c->ilu_diag); dfree(c->ilu_rowmap); }
    c->ilu_rowmap = nullptr;
    c->ilu_owns_pattern = false;
    c->ilu_rp = c->ilu_ci = c->ilu_diag = nullptr;
    dfree(c->lvl_f); dfree(c->lvl_b); dfree(c->LU); dfree(c->ybuf); dfree(c->zbuf);
    c->lvl_f = c->lvl_b = nullptr;
    c->LU = c->ybuf = c->zbuf = nullptr;
    void **sf[] = {(void **)&c->sf_pos_f, (void **)&c->sf_pos_b, (void **)&c->sf_bmap, (void **)&c->sf_off_f,
                   (void **)&c->sf_off_b, (void **)&c->sf_col_f, (void **)&c->sf_col_b, (void **)&c->sf_val_f,
                   (void **)&c->sf_val_b, (void **)&c->sf_dinv, (void **)&c->sf_ticket, (void **)&c->sf_y,
                   (void **)&c->sf_z, (void **)&c->sp_inv_f, (void **)&c->sp_inv_b, (void **)&c->sp_levr_f,
                   (void **)&c->sp_levr_b};
    for (void **p : sf) { dfree(*p); *p = nullptr; }
    pair_free(c);
    c->sp_use = false;
}

// launch one chunked sweep with its tables (NS = stage slots chosen at set-up)
template <int B, typename T, typename ST, typename XT, bool FWD>
static void cw_launch(const Ctx *c, const CwTables &t, const ST *src, T *vec, double *out, const XT *dp, const XT *dT,
                      const double *never) {
    const unsigned grid = (unsigned)std::min(t.nchunks, 152);
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, t.smem);
        cudaMemsetAsync(t.started, 0, sizeof(int32_t) * t.nchunks, c->stream);
        (kern<<<grid, t.threads, t.smem, c->stream>>>(t.nchunks, c->n, t.D, t.W, t.maxw, t.maxlev, c->sf_ticket, t.clev,
                                                     t.lptr, t.prow, t.code, (const T *)t.val, src, vec, out, c->ps,
                                                     c->ts, dp, dT, c->ks, never, c->sf_sleep, t.started, kCwLead),
         note_launch());
    };
    if (t.ns == 3) go(k_ilu_cw<B, T, ST, XT, FWD, 3>);
    else if (t.ns == 2) go(k_ilu_cw<B, T, ST, XT, FWD, 2>);
    else go(k_ilu_cw<B, T, ST, XT, FWD, 1>);
}

// z = (LU)^{-1} r + x1, where x1 carries dp in slot ps and dT in slot ts (either may be null):
// sentinel fill, forward sweep, backward sweep (three launches).  T: factor storage and sweep
// arithmetic; RT: type of r; XT: type of dp, dT.
template <int B, typename T, typename RT, typename XT>
static void sweeps(const Ctx *c, const RT *r, double *z, const XT *dp, const XT *dT) {
    cudaStream_t s = c->stream;
    const int32_t n = c->n;
    T *y = (T *)c->sf_y, *zz = (T *)c->sf_z;
    (k_sf_fill<T><<<4 * 152, 256, 0, s>>>((int64_t)n * B, y, zz, c->sf_ticket), note_launch());
    if (c->inject_wait) (k_sf_fill<double><<<1, 32, 0, s>>>(1, c->never, c->never, c->sf_ticket + 2), note_launch());
    if (c->tl_use) {
        tile_apply<T, RT, XT>(c, r, z, dp, dT);
        return;
    }
    if (c->cw_use) {
        const CwTables &F = c->cw_f, &Bk = c->cw_b;
        int pf = prof_begin(c, PF_ILU_FWD);
        cw_launch<B, T, RT, XT, true>(c, F, r, y, nullptr, nullptr, nullptr, c->inject_wait ? c->never : nullptr);
        prof_end(c, pf);
        pf = prof_begin(c, PF_ILU_BWD);
        cw_launch<B, T, T, XT, false>(c, Bk, y, zz, z, dp, dT, nullptr);
        prof_end(c, pf);
        return;
    }
    if (c->sp_use && c->sf_half >= 2) {   // grouped levels, a row over 8 or 16 lanes (2 or 4 parts)
        const unsigned gridh = std::min<unsigned>(nblk(n, kSfThreads / (kSfGroup * c->sf_half)), (unsigned)c->sf_grid);
        int pf = prof_begin(c, PF_ILU_FWD);
        auto fwd = [&](auto kern) {
            (kern<<<gridh, kSfThreads, 0, s>>>(n, c->sf_ticket, c->sf_pos_f, c->sp_off_f, c->sp_col_f,
                                               (const T *)c->sp_val_f, r, y, c->ks, c->inject_wait ? c->never : nullptr,
                                               c->sf_sleep, c->sp_coff_f, c->sp_ccol_f, (const T *)c->sp_cval_f),
             note_launch());
        };
        if (c->sf_half == 4) fwd(k_ilu_fwd_h<B, T, RT, 3, 4>);
        else if (c->sp_group >= 3) fwd(k_ilu_fwd_h<B, T, RT, 6, 2>);
        else fwd(k_ilu_fwd_h<B, T, RT, 4, 2>);
        prof_end(c, pf);
        pf = prof_begin(c, PF_ILU_BWD);
        auto bwd = [&](auto kern) {
            (kern<<<gridh, kSfThreads, 0, s>>>(n, c->sf_ticket, c->sf_pos_b, c->sf_bmap, c->sp_off_b, c->sp_col_b,
                                               (const T *)c->sp_val_b, (const T *)c->sf_dinv, y, zz, z, c->ps, c->ts, dp,
                                               dT, c->ks, c->sf_sleep, c->sp_coff_b, c->sp_ccol_b,
                                               (const T *)c->sp_cval_b),
             note_launch());
        };
        if (c->sf_half == 4) bwd(k_ilu_bwd_h<B, T, XT, 3, 4>);
        else if (c->sp_group >= 3) bwd(k_ilu_bwd_h<B, T, XT, 6, 2>);
        else bwd(k_ilu_bwd_h<B, T, XT, 4, 2>);
        prof_end(c, pf);
        return;
    }
    if (std::is_same<T, double>::value || c->sp_use) {   // a row over four lanes, lockstep rounds
        const unsigned gridg = std::min<unsigned>(nblk(n, kSfRowsG), (unsigned)c->sf_grid);
        // the level-set tables, or the paired-level ones (their c-term tables non-null)
        const bool pr = c->sp_use;
        int pf = prof_begin(c, PF_ILU_FWD);
        auto fwd = [&](auto kern) {
            (kern<<<gridg, kSfThreads, 0, s>>>(
                 n, c->sf_ticket, c->sf_pos_f, pr ? c->sp_off_f : c->sf_off_f, pr ? c->sp_col_f : c->sf_col_f,
                 pr ? (const T *)c->sp_val_f : (const T *)c->sf_val_f, r, y, c->ks,
                 c->inject_wait ? c->never : nullptr, c->sf_sleep, pr ? c->sp_coff_f : nullptr, c->sp_ccol_f,
                 (const T *)c->sp_cval_f),
             note_launch());
        };
        if (pr && c->sp_group >= 3) fwd(k_ilu_fwd_g<B, T, RT, 12>);
        else if (pr) fwd(k_ilu_fwd_g<B, T, RT, 8>);
        else fwd(k_ilu_fwd_g<B, T, RT, kDepGroup>);
        prof_end(c, pf);
        pf = prof_begin(c, PF_ILU_BWD);
        auto bwd = [&](auto kern) {
            (kern<<<gridg, kSfThreads, 0, s>>>(
                 n, c->sf_ticket, c->sf_pos_b, c->sf_bmap, pr ? c->sp_off_b : c->sf_off_b,
                 pr ? c->sp_col_b : c->sf_col_b, pr ? (const T *)c->sp_val_b : (const T *)c->sf_val_b,
                 (const T *)c->sf_dinv, y, zz, z, c->ps, c->ts, dp, dT, c->ks, c->sf_sleep,
                 pr ? c->sp_coff_b : nullptr, c->sp_ccol_b, (const T *)c->sp_cval_b),
             note_launch());
        };
        if (pr && c->sp_group >= 3) bwd(k_ilu_bwd_g<B, T, XT, 12, true>);
        else if (pr) bwd(k_ilu_bwd_g<B, T, XT, 8, true>);
        else bwd(k_ilu_bwd_g<B, T, XT, kDepGroup>);
        prof_end(c, pf);
        return;
    }
    const unsigned grid = std::min<unsigned>(nblk(n, kSfThreads), (unsigned)c->sf_grid);
    int pf = prof_begin(c, PF_ILU_FWD);
    (k_ilu_fwd_sf<B, T, RT><<<grid, kSfThreads, 0, s>>>(n, c->sf_ticket, c->sf_pos_f, c->sf_off_f, c->sf_col_f,
                                                         (const T *)c->sf_val_f, r, y, c->ks,
                                                         c->inject_wait ? c->never : nullptr, c->sf_sleep), note_launch());
    prof_end(c, pf);
    pf = prof_begin(c, PF_ILU_BWD);
    (k_ilu_bwd_sf<B, T, XT><<<grid, kSfThreads, 0, s>>>(n, c->sf_ticket, c->sf_pos_b, c->sf_bmap, c->sf_off_b,
                                                         c->sf_col_b, (const T *)c->sf_val_b, (const T *)c->sf_dinv, y,
                                                         zz, z, c->ps, c->ts, dp, dT, c->ks, c->sf_sleep), note_launch());
    prof_end(c, pf);
}

void ilu_apply(const Ctx *c, const double *r, double *z, const double *dp, const double *dT) {
    if (c->o.precision == CPTR_PREC_MIXED) {
        if (c->b == 3) sweeps<3, float, double, double>(c, r, z, dp, dT);
        else sweeps<4, float, double, double>(c, r, z, dp, dT);
    } else {
        if (c->b == 3) sweeps<3, double, double, double>(c, r, z, dp, dT);
        else sweeps<4, double, double, double>(c, r, z, dp, dT);
    }
}

// mixed-precision form: r, dp, dT in FP32, factors FP32, z FP64
void ilu_apply32(const Ctx *c, const float *r, double *z, const float *dp, const float *dT) {
    if (c->b == 3) sweeps<3, float, float, float>(c, r, z, dp, dT);
    else sweeps<4, float, float, float>(c, r, z, dp, dT);
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

// Autotuner of the one-launch ILU(0) sweeps: the persistent grid (blocks in {152, 304, 608,
// 1216}) and the back-off between polls of a dependency not yet written (__nanosleep of {0, 8, 32,
// 128, 512} ns), which set how many rows run ahead of the wavefront and how hard they poll, for
// the level-set schedule and, where they were built, the paired-level one; the back-off of the
// chunked schedule; the fastest schedule is kept.  Each candidate is timed with CUDA events over 3
// applications (forward + backward) after a warm-up, on a zero right-hand side; the result is
// cached by the factor size.
cptr_status ilu_autotune(Ctx *c) {
    if (!c->LU) return CPTR_OK;
    const uint64_t key = ilu_tune_key(c);
    const bool auto_sched = c->o.ilu_sweep == 0;
    auto it = c->tune_cache.find(key);
    if (it != c->tune_cache.end()) {
        c->sf_grid = it->second.T;
        c->sf_sleep = it->second.G;
        auto hf = c->tune_cache.find(key + 3);
        c->sf_half = c->o.ilu_lanes ? c->o.ilu_lanes / 4 : (hf != c->tune_cache.end() ? hf->second.G : 1);
        if (auto_sched) {
            const int sched = ilu_tuned_schedule(c);
            c->cw_use = c->cw_ok && sched == 1;
            c->sp_use = c->sp_ok && sched == 2;
            c->tl_use = c->tl_ok && sched == 3;
        }
        auto ts = c->tune_cache.find(key + 2);
        if (ts != c->tune_cache.end()) { c->tl_best_ty = ts->second.G; c->tl_best_tz = ts->second.T; }
        return CPTR_OK;
    }
    double *r = c->xw, *z = c->w;   // scratch vectors of n*b doubles
    const bool cw_was = c->cw_use, sp_was = c->sp_use, tl_was = c->tl_use;
    c->cw_use = false;              // time the level-set sweeps first (or the paired ones if forced)
    c->sp_use = c->sp_ok && c->o.ilu_sweep == 3;
    c->tl_use = false;
    CPTR_CUDA_TRY(c, cudaMemsetAsync(r, 0, sizeof(double) * (size_t)c->n * c->b, c->stream));
    cudaEvent_t e0, e1;
    CPTR_CUDA_TRY(c, cudaEventCreate(&e0));
    CPTR_CUDA_TRY(c, cudaEventCreate(&e1));
    auto time3 = [&]() -> float {   // one warm-up, then 3 applications
        ilu_apply(c, r, z, nullptr, nullptr);
        cudaEventRecord(e0, c->stream);
        for (int rep = 0; rep < 3; ++rep) ilu_apply(c, r, z, nullptr, nullptr);
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    const unsigned maxg = nblk(c->n, kSfThreads);
    // grid x back-off of the schedule now set; the fastest pair and its time
    auto search = [&](int *bg, int *bs) -> float {
        float bm = 1e30f;
        for (int g : {152, 304, 608, 1216}) {
            if (g > (int)maxg && g != 152) continue;
            for (int sl : {0, 8, 32, 128, 512}) {
                c->sf_grid = g;
                c->sf_sleep = sl;
                const float ms = time3();
                if (ms < bm) { bm = ms; *bg = g; *bs = sl; }
            }
        }
        return bm;
    };
    int best_g = c->sf_grid, best_s = c->sf_sleep;
    const int fixed_half = c->o.ilu_lanes / 4;   // 0: both are timed
    c->sf_half = fixed_half ? fixed_half : 1;
    float best_ms = search(&best_g, &best_s);
    int best_half = c->sf_half;   // grouped levels: a row over four lanes, or over eight (two halves)
    if (c->sp_use && !fixed_half) {
        for (int hf : {2, 4}) {
            c->sf_half = hf;
            int g = best_g, sl = best_s;
            const float ms = search(&g, &sl);
            if (ms < best_ms) { best_ms = ms; best_g = g; best_s = sl; best_half = hf; }
        }
        c->sf_half = 1;
    }
    int sched = c->sp_use ? 2 : 0;
    int group = c->sp_use ? c->sp_group : 0;
    // the other schedules, each at its own best grid and back-off; the fastest is kept
    // grouped levels: groups of two (the tables built at set-up) and, unless the caller fixed the
    // group size, of three (tables rebuilt for the timing), each over 4, 8 and 16 lanes per row.
    // Groups of three cost more set-up (their tables hold products of three factor blocks), so
    // they are kept only when their sweeps are at least 5% faster than the best so far.
    if (auto_sched && c->sp_ok) {
        const int g0 = c->sp_group;
        const int ng = (c->o.ilu_group >= 2 || g0 == 3) ? 1 : 2;
        int bgroup = 0;
        for (int gi = 0; gi < ng; ++gi) {
            const int G = gi == 0 ? g0 : 3;
            if (gi > 0) {
                CPTR_TRY(pair_setup(c, G));
                if (!c->sp_ok) break;
            }
            const float need = G == g0 ? 1.0f : 0.95f;
            c->sp_use = true;
            for (int hf : {1, 2, 4}) {
                if (fixed_half && hf != fixed_half) continue;
                c->sf_half = hf;
                int g = best_g, sl = best_s;
                const float ms = search(&g, &sl);
                if (ms < need * best_ms) {
                    best_ms = ms; best_g = g; best_s = sl; sched = 2; group = G; best_half = hf; bgroup = G;
                }
            }
            c->sf_half = 1;
            c->sp_use = false;
        }
        const int keep = bgroup ? bgroup : g0;
        if (c->sp_group != keep || !c->sp_ok) CPTR_TRY(pair_setup(c, keep));
    }
    if (auto_sched && c->cw_ok) {   // one block per chunk: only the back-off matters
        c->cw_use = true;
        float bm = 1e30f;
        int sl = best_s;
        for (int v : {0, 8, 32, 128, 512}) {
            c->sf_sleep = v;
            const float ms = time3();
            if (ms < bm) { bm = ms; sl = v; }
        }
        c->cw_use = false;
        if (bm < best_ms) { best_ms = bm; best_s = sl; sched = 1; }
    }
    // tiled sweeps: the back-off, and the tile shapes of smallest modelled time (the tables are
    // rebuilt for each shape timed; the fastest shape's tables are kept)
    int tile_ty = 0, tile_tz = 0;
    if ((auto_sched || c->o.ilu_sweep == 4) && c->tl_dims[0]) {
        std::vector<std::pair<int, int>> cand;
        if (c->o.tile_y > 0 || c->o.tile_z > 0) {
            if (c->tl_ok) cand.push_back({c->tl_ty, c->tl_tz});   // the caller's shape only
        } else {
            tile_candidates(c, 4, cand);
        }
        float bt = 1e30f;
        int bsl = best_s;
        for (const auto &sh : cand) {
            CPTR_TRY(tile_setup(c, sh.first, sh.second));
            if (!c->tl_ok) continue;
            c->tl_use = true;
            for (int v : {0, 32, 128}) {
                c->sf_sleep = v;
                const float ms = time3();
                if (ms < bt) { bt = ms; bsl = v; tile_ty = sh.first; tile_tz = sh.second; }
            }
            c->tl_use = false;
        }
        if (tile_ty > 0) {
            if (c->tl_ty != tile_ty || c->tl_tz != tile_tz) CPTR_TRY(tile_setup(c, tile_ty, tile_tz));
            if (auto_sched && bt < best_ms) { best_ms = bt; best_s = bsl; sched = 3; }
            if (c->o.ilu_sweep == 4) { best_s = bsl; sched = 3; }
        }
    }
    c->sf_grid = best_g;
    if (auto_sched) {
        c->cw_use = sched == 1;
        c->sp_use = sched == 2;
        c->tl_use = sched == 3 && c->tl_ok;
    } else {
        c->cw_use = cw_was;
        c->sp_use = sp_was;
        c->tl_use = tl_was && c->tl_ok;
    }
    c->sf_sleep = best_s;
    c->sf_half = c->sp_use ? best_half : 1;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    Shape sh, sc;
    sh.T = (int16_t)best_g;
    sh.G = (int16_t)best_s;
    sc.G = (int16_t)sched;
    sc.T = (int16_t)(sched == 2 ? group : 0);
    c->tune_cache[key] = sh;
    c->tune_cache[key + 1] = sc;
    Shape hs;
    hs.G = (int16_t)c->sf_half;
    hs.T = 0;
    c->tune_cache[key + 3] = hs;
    if (tile_ty > 0) {
        c->tl_best_ty = tile_ty;
        c->tl_best_tz = tile_tz;
        Shape st;
        st.G = (int16_t)tile_ty;
        st.T = (int16_t)tile_tz;
        c->tune_cache[key + 2] = st;
    }
    CPTR_CUDA_TRY(c, cudaGetLastError());
    return CPTR_OK;
}

}  // namespace cptr
