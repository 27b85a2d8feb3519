// Tiled ILU(0) triangular sweeps (the second stage's z = (LU)^{-1} r, Sec. 3 two-stage step 3 and
// Sec. 4), an evaluation order of the same solves as the level-set sweeps of ilu.cu: every value
// is computed with the same operations in the same order, so results are bit-identical.
//
// On a Cartesian box in natural order (cell x + nx (y + ny z)) the rows of a grid line (fixed y, z)
// are consecutive and each depends on the one before.  The lines are grouped into tiles of
// Ty x Tz lines; one block owns a tile and walks the tile's own level sets (levels counted over
// dependencies inside the tile, x + (y - y0) + (z - z0) on the box), with one __syncthreads per
// level and the tile's solved values kept in a shared-memory ring.  Only dependencies on another
// tile (the tile's faces at y0 - 1 and z0 - 1) go through global memory; their values are polled
// (the sentinel of sweep.cuh, bounded waits), and since a tile starts only once its upstream
// tiles have produced the rows it needs, it trails them by a few levels and finds those values
// already written.  A sweep's dependency chain thus costs ny/Ty + nz/Tz cross-block hops plus
// nx + Ty + Tz in-block levels, instead of nx + ny + nz cross-block steps.
//
// Per position (rows tile by tile in processing order, by local level inside a tile) a record
// holds the row, its dependency codes (a ring slot, or the global row of a value to poll) and its
// factor blocks (and, backward, the inverted pivot block).  The records of a level are one
// contiguous run, copied into shared memory by a TMA bulk copy (cp.async.bulk completing on an
// mbarrier) 2P levels ahead; P levels ahead, each row's right-hand side and the 16-byte
// windows around its outside dependencies' values are copied by cp.async (through L2 only), so
// that a level starts with everything in shared memory.  A value copied before it was written
// holds the sentinel and is polled from global memory when used.
//
// Tiles are handed out by a ticket in an order where every outside dependency lies in an earlier
// tile, so a block only waits on tiles held by blocks that already run: no deadlock, whatever
// the grid.  Every wait (a polled value, an mbarrier) is bounded.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>
#include <vector>

#include "common.cuh"
#include "sweep.cuh"

namespace cptr {

namespace {

constexpr int32_t kTileNone = INT32_MIN;   // no dependency in this slot
constexpr int kTileMaxRows = 64;           // rows of one level of a tile (4 lanes each: <= 256 threads)
constexpr int kTileWin = 48;               // bytes of the 16-byte-aligned window around a row's value
constexpr int kTileBar = 256;              // shared-memory bytes reserved for the mbarriers
constexpr size_t kTileSmemMax = 200 * 1024;

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// record: int32 row, int32 code[D], padded to 16 bytes; T blk[D][B*B] (backward: then T dinv[B*B]),
// padded to 16 bytes
__host__ __device__ inline int hdr_bytes(int D) { return ((1 + D) * 4 + 15) & ~15; }
__host__ __device__ inline int rec_bytes(int D, int BB, int tsz, bool fwd) {
    return hdr_bytes(D) + (((D + (fwd ? 0 : 1)) * BB * tsz + 15) & ~15);
}
// staged inputs of one row: its right-hand side (B values, padded to 16 bytes), the backward
// sweep's x1 terms (B doubles: lane ps holds dp, lane ts holds dT), one window per slot
__host__ __device__ inline int rhs_bytes(int B, int ssz) { return ((B * ssz + 15) & ~15) + ((B * 8 + 15) & ~15); }
__host__ __device__ inline int val_bytes(int D, int B, int ssz) { return rhs_bytes(B, ssz) + D * kTileWin; }
// shared-memory bytes of a tile's level pointers
__host__ __device__ inline int lv_bytes(int maxnl) { return ((maxnl + 1) * 4 + 15) & ~15; }

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *m, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *m, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *m, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(m)), "r"(parity)
        : "memory");
    return ok != 0;
}
// TMA bulk copy global -> shared, completing on the mbarrier (16-byte aligned, multiple of 16 bytes)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *m) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(m))
                 : "memory");
}
__device__ __forceinline__ void cp_async_cg16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_ca(double *dst, const double *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_ca(float *dst, const float *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
// the x1 term of a row (dp or dT, FP64 or FP32) into a staged double slot; read back by x1_value
__device__ __forceinline__ void cp_async_x1(double *dst, const double *src) { cp_async_ca(dst, src); }
__device__ __forceinline__ void cp_async_x1(double *dst, const float *src) {
    cp_async_ca(reinterpret_cast<float *>(dst), src);
}
__device__ __forceinline__ double x1_value(const double *slot, const double *) { return *slot; }
__device__ __forceinline__ double x1_value(const double *slot, const float *) {
    return (double)*reinterpret_cast<const float *>(slot);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// a bounded wait of this call has given up (relaxed GPU-scope read of the flag)
__device__ __forceinline__ bool failed(KState *ks) {
    int32_t f;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(f) : "l"(&ks->wait_err) : "memory");
    return f != 0;
}

// bounded wait for the records of a level (parity of the stage's use); false if it gave up
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *m, unsigned parity) {
    if (mbar_try_wait(m, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (;;) {
        if (mbar_try_wait(m, parity)) return true;
        if (gtimer() - t0 > kWaitNs) return false;
    }
}

// One sweep.  Forward (FWD): y(row) = r(row) - sum_d L(row, d) y(dep d).  Backward:
// z(row) = D(row)^{-1} (y(row) - sum_d U(row, d) z(dep d)), out(row) = z(row) + x1(row), x1 carrying
// dp in slot ps and dT in slot ts.  src: r (forward, type ST) or y (backward); vec: the vector being
// solved, in row order.
//
// Warp-specialised: the last warp of the block is the producer, the others are consumers.  Lane q
// of a consumer row group of four computes component q (B <= 4), like the four-lane level-set
// kernels; the consumers only read shared memory and do the level's arithmetic, one named barrier
// per level among themselves.  The producer runs P levels ahead: at its step m it copies the
// records of level m + P (TMA bulk copy onto rec_full), waits for the records of level m, and
// copies each row's right-hand side, x1 terms and outside-dependency windows (cp.async, completion
// tracked by cp.async.mbarrier.arrive on val_full).  Consumers release a value slot (val_empty)
// when they finish its level; that also frees the record stage the producer refills next, since
// NS = 2P + 1 stages and NV = P + 1 value slots are in flight.
template <int B, typename T, typename ST, typename XT, bool FWD, int P>
__global__ void __launch_bounds__(4 * kTileMaxRows + 32)
    k_ilu_tile(int32_t ntiles, const int32_t *__restrict__ tlev, const int32_t *__restrict__ lptr,
               const unsigned char *__restrict__ rec, int RS, int D, int R, int MW, int maxnl,
               const ST *__restrict__ src, T *vec, double *__restrict__ out, int ps, int ts,
               const XT *__restrict__ dp, const XT *__restrict__ dT, unsigned *ticket, KState *ks,
               const double *never, int sleep_ns) {
    constexpr int BB = B * B, NS = 2 * P + 1, NV = P + 1;
    constexpr int WPIECES = (8 * B + 15 + 15) / 16;   // 16-byte pieces of a window (value + skew)
    const int H = hdr_bytes(D), RH = rhs_bytes(B, (int)sizeof(ST)), SV = val_bytes(D, B, (int)sizeof(ST));
    const int XA = (B * (int)sizeof(ST) + 15) & ~15;   // offset of the x1 terms in a staged row
    extern __shared__ __align__(128) unsigned char tile_smem[];
    uint64_t *rec_full = reinterpret_cast<uint64_t *>(tile_smem);
    uint64_t *val_full = rec_full + NS;
    uint64_t *val_empty = val_full + NV;
    int32_t *lv = reinterpret_cast<int32_t *>(tile_smem + kTileBar);   // the tile's level pointers
    unsigned char *recs = tile_smem + kTileBar + lv_bytes(maxnl);
    unsigned char *vals = recs + (size_t)NS * MW * RS;
    T *ring = reinterpret_cast<T *>(vals + (size_t)NV * MW * SV);
    __shared__ unsigned tile_s;
    __shared__ volatile int abort_s;   // a bounded wait gave up: every wait returns at once
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ncons = (int)blockDim.x - 32;   // consumer threads; the producer is the last warp
    const bool producer = tid >= ncons;
    const int g = tid >> 2, q4 = tid & 3;
    const int g0 = (tid & 31) & ~3;
    const unsigned gmask = ((1u << B) - 1u) << g0;
    (void)warp;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&rec_full[s], 1);
        for (int s = 0; s < NV; ++s) {
            mbar_init(&val_full[s], 32);
            mbar_init(&val_empty[s], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        abort_s = 0;
    }
    __syncthreads();
    // bounded wait on an mbarrier phase; gives up at once when this call has already failed
    auto wait_bar = [&](uint64_t *m, unsigned parity) {
        if (mbar_try_wait(m, parity)) return;
        const unsigned long long t0 = gtimer();
        for (;;) {
            if (mbar_try_wait(m, parity)) return;
            const unsigned long long dt = gtimer() - t0;
            if (dt > kWaitNs || abort_s || (dt > 100000ull && failed(ks))) {
                atomicExch(&ks->wait_err, 1);
                abort_s = 1;
                return;
            }
        }
    };
    unsigned gl = 0;   // levels this block has processed: stage indices and mbarrier phases
    for (;;) {
        if (tid == 0) tile_s = atomicAdd(ticket + (FWD ? 0 : 1), 1u);
        __syncthreads();
        const unsigned tile = tile_s;
        if (tile >= (unsigned)ntiles || abort_s) break;
        const int L0 = __ldg(tlev + tile), nl = __ldg(tlev + tile + 1) - L0;
        for (int q = tid; q <= nl; q += blockDim.x) lv[q] = __ldg(lptr + L0 + q);
        __syncthreads();
        const int32_t pos0 = lv[0];
        if (producer) {
            int issued = 0;   // record stages issued (lane 0)
            auto issue_rec = [&](int m) {
                const unsigned G = gl + m;
                const unsigned bytes = (unsigned)(lv[m + 1] - lv[m]) * (unsigned)RS;
                mbar_expect_tx(&rec_full[G % NS], bytes);
                bulk_g2s(recs + (size_t)(G % NS) * MW * RS, rec + (size_t)lv[m] * RS, bytes, &rec_full[G % NS]);
                ++issued;
            };
            if (lane == 0)
                for (int m = 0; m < min(P, nl); ++m) issue_rec(m);
            for (int m = 0; m < nl && !abort_s; ++m) {
                const unsigned G = gl + m;
                if (G >= (unsigned)NV) wait_bar(&val_empty[G % NV], (G / NV - 1) & 1u);   // level G - NV done
                if (lane == 0 && m + P < nl) issue_rec(m + P);   // its stage's last level was G - NV
                wait_bar(&rec_full[G % NS], (G / NS) & 1u);
                const int w = lv[m + 1] - lv[m];
                for (int r0 = lane; r0 < w; r0 += 32) {
                    const unsigned char *r = recs + (size_t)(G % NS) * MW * RS + (size_t)r0 * RS;
                    const int32_t row = *reinterpret_cast<const int32_t *>(r);
                    const int32_t *code = reinterpret_cast<const int32_t *>(r) + 1;
                    unsigned char *dst = vals + ((size_t)(G % NV) * MW + r0) * SV;
#pragma unroll
                    for (int q = 0; q < B; ++q) cp_async_ca(reinterpret_cast<ST *>(dst) + q, src + (int64_t)row * B + q);
                    if (!FWD) {
                        double *xa = reinterpret_cast<double *>(dst + XA);
                        if (dp) cp_async_x1(xa + ps, dp + row);
                        if (dT) cp_async_x1(xa + ts, dT + row);
                    }
                    for (int d = 0; d < D; ++d) {
                        const int32_t cd = code[d];
                        if (cd == kTileNone) break;
                        if (cd >= 0) continue;
                        const int64_t j = -(int64_t)cd - 1;
                        const uintptr_t at = reinterpret_cast<uintptr_t>(vec + j * B) & ~(uintptr_t)15;
#pragma unroll
                        for (int k = 0; k < WPIECES; ++k)
                            cp_async_cg16(dst + RH + d * kTileWin + 16 * k, reinterpret_cast<const void *>(at + 16 * k));
                    }
                }
                asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&val_full[G % NV]))
                             : "memory");
            }
            asm volatile("cp.async.wait_all;" ::: "memory");
            if (abort_s && lane == 0)   // record copies still in flight: wait (bounded) for them
                for (int m = 0; m < issued; ++m) {
                    const unsigned G = gl + m;
                    (void)mbar_wait_bounded(&rec_full[G % NS], (G / NS) & 1u);
                }
        } else {
            for (int l = 0; l < nl; ++l) {
                const unsigned G = gl + l;
                // after a failed wait the consumers still pass every level's barrier together
                wait_bar(&val_full[G % NV], (G / NV) & 1u);
                wait_bar(&rec_full[G % NS], (G / NS) & 1u);
                const int w = abort_s ? 0 : lv[l + 1] - lv[l];
                const int32_t p0 = lv[l] - pos0;   // local position of the level's first row
                if (g < w && q4 < B) {
                    const unsigned char *r = recs + (size_t)(G % NS) * MW * RS + (size_t)g * RS;
                    const int32_t row = *reinterpret_cast<const int32_t *>(r);
                    const int32_t *code = reinterpret_cast<const int32_t *>(r) + 1;
                    const T *blk = reinterpret_cast<const T *>(r + H);
                    const unsigned char *vb = vals + ((size_t)(G % NV) * MW + g) * SV;
                    if (FWD && never && tile == 0 && l == 0 && g == 0 && q4 == 0) (void)wait_value(never, ks);
                    T acc = (T) reinterpret_cast<const ST *>(vb)[q4];
                    for (int d = 0; d < D; ++d) {
                        const int32_t cd = code[d];
                        if (cd == kTileNone) break;
                        T v[B];
                        if (cd >= 0) {
#pragma unroll
                            for (int u = 0; u < B; ++u) v[u] = ring[cd * B + u];
                        } else {
                            const uint32_t j32 = (uint32_t)(-(cd + 1));
                            const T *win = reinterpret_cast<const T *>(vb + RH + d * kTileWin +
                                                                       ((j32 * (uint32_t)(B * sizeof(T))) & 15u));
                            bool pend = false;
#pragma unroll
                            for (int u = 0; u < B; ++u) {
                                v[u] = win[u];
                                pend |= is_sentinel(v[u]);
                            }
                            if (pend) {   // copied before it was written: poll (bounded)
                                const int64_t j = (int64_t)j32;
                                const unsigned long long t0 = gtimer();
                                for (;;) {
                                    pend = false;
#pragma unroll
                                    for (int u = 0; u < B; ++u)
                                        if (is_sentinel(v[u])) {
                                            v[u] = load_relaxed(vec + j * B + u);
                                            pend |= is_sentinel(v[u]);
                                        }
                                    if (!pend) break;
                                    const unsigned long long dt = gtimer() - t0;
                                    // give up after kWaitNs, or after 100 us once any wait of the
                                    // call has given up (its values will not come)
                                    if (dt > kWaitNs || (dt > 100000ull && failed(ks))) {
                                        atomicExch(&ks->wait_err, 1);
                                        abort_s = 1;
#pragma unroll
                                        for (int u = 0; u < B; ++u)
                                            if (is_sentinel(v[u])) v[u] = (T)0;
                                        break;
                                    }
                                    __nanosleep(sleep_ns);
                                }
                            }
                        }
#pragma unroll
                        for (int u = 0; u < B; ++u) acc = fma(-blk[d * BB + q4 * B + u], v[u], acc);
                    }
                    T res;
                    if (FWD) {
                        res = acc;
                    } else {
                        const T *dinv = blk + D * BB;
                        res = (T)0;
#pragma unroll
                        for (int u = 0; u < B; ++u) res = fma(dinv[q4 * B + u], __shfl_sync(gmask, acc, g0 + u), res);
                    }
                    ring[((p0 + g) & (R - 1)) * B + q4] = res;
                    store_relaxed(vec + (int64_t)row * B + q4, res);
                    if (!FWD) {
                        const double *xa = reinterpret_cast<const double *>(vb + XA);
                        double add = 0.0;
                        if (dp && q4 == ps) add = x1_value(xa + q4, dp);
                        if (dT && q4 == ts) add = x1_value(xa + q4, dT);
                        out[(int64_t)row * B + q4] = (double)res + add;
                    }
                }
                // the level's ring values are visible to every consumer, and its slots are free
                asm volatile("bar.sync 1, %0;" ::"r"(ncons) : "memory");
                if (tid == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&val_empty[G % NV]))
                                           : "memory");
            }
        }
        __syncthreads();
        if (abort_s) break;
        gl += (unsigned)nl;
    }
}

// records of one sweep: header (row, codes) from hdr[p][1 + D], blocks from LU by kidx[p][D (+1)]
template <typename T>
__global__ void k_tile_pack(int32_t n, int D, int BB, int RS, int H, int nslot, const int32_t *__restrict__ hdr,
                            const int32_t *__restrict__ kidx, const double *__restrict__ LU, unsigned char *rec) {
    const int32_t p = (int32_t)(blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
    if (p >= n) return;
    unsigned char *r = rec + (size_t)p * RS;
    int32_t *h = reinterpret_cast<int32_t *>(r);
    for (int e = 0; e < H / 4; ++e) h[e] = e <= D ? hdr[(size_t)p * (1 + D) + e] : 0;
    T *blk = reinterpret_cast<T *>(r + H);
    for (int d = 0; d < nslot; ++d) {
        const int32_t k = kidx[(size_t)p * nslot + d];
        for (int e = 0; e < BB; ++e) blk[d * BB + e] = k >= 0 ? (T)LU[(size_t)k * BB + e] : (T)0;
    }
    for (int e = nslot * BB * (int)sizeof(T); e < RS - H; ++e) r[H + e] = 0;
}

// run f(t) for t in [0, count) on up to 8 host threads
template <typename F>
void parallel_for(int32_t count, F &&f) {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nt = (int)std::min<unsigned>(std::min<unsigned>(8u, hw), (unsigned)std::max(count, 1));
    if (nt <= 1) {
        for (int32_t t = 0; t < count; ++t) f(t);
        return;
    }
    std::atomic<int32_t> next(0);
    std::vector<std::thread> pool;
    for (int i = 0; i < nt; ++i)
        pool.emplace_back([&]() {
            for (int32_t t = next++; t < count; t = next++) f(t);
        });
    for (auto &th : pool) th.join();
}

// host tables of one sweep for tiles of Ty x Tz lines: positions, level pointers, record headers
// and block indices; false when the schedule does not apply (a level wider than kTileMaxRows, or an
// outside dependency on a later tile)
struct TileHost {
    int32_t ntiles = 0, nlev = 0, D = 0, MW = 0, maxnl = 0;
    std::vector<int32_t> tlev, lptr, hdr, kidx;
};

bool tile_build(int32_t n, const std::vector<int32_t> &rp, const std::vector<int32_t> &ci,
                const std::vector<int32_t> &dg, const int32_t dims[3], int Ty, int Tz, bool fwd, int R,
                TileHost &h) {
    const int32_t nx = dims[0], ny = dims[1], nz = dims[2];
    const int32_t nty = (ny + Ty - 1) / Ty, ntz = (nz + Tz - 1) / Tz, nt = nty * ntz;
    auto dep = [fwd](int32_t i, int32_t j) { return fwd ? j < i : j > i; };
    // processing order of the tiles: by ty + tz (ascending forward, descending backward), then tz
    std::vector<int32_t> order(nt), rank(nt);
    for (int32_t t = 0; t < nt; ++t) order[t] = t;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        const int32_t sa = a % nty + a / nty, sb = b % nty + b / nty;
        if (sa != sb) return fwd ? sa < sb : sa > sb;
        return fwd ? a < b : a > b;
    });
    for (int32_t k = 0; k < nt; ++k) rank[order[k]] = k;
    std::vector<int32_t> tile_of(n);
    std::vector<int32_t> cnt(nt + 1, 0);
    int32_t D = 0;
    for (int32_t i = 0; i < n; ++i) {
        const int32_t y = (i / nx) % ny, z = i / (nx * ny);
        tile_of[i] = rank[(z / Tz) * nty + y / Ty];
        ++cnt[tile_of[i] + 1];
        int32_t nd = 0;
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) nd += dep(i, ci[k]) ? 1 : 0;
        D = std::max(D, nd);
    }
    for (int32_t t = 0; t < nt; ++t) cnt[t + 1] += cnt[t];
    // rows of each tile in sweep order (ascending forward, descending backward)
    std::vector<int32_t> rows(n);
    {
        std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
        for (int32_t u = 0; u < n; ++u) {
            const int32_t i = fwd ? u : n - 1 - u;
            rows[fill[tile_of[i]]++] = i;
        }
    }
    std::vector<int32_t> lev(n, 0), lpos(n, 0), nlev_t(nt, 0), width_t(nt, 0);
    std::vector<std::vector<int32_t>> lcount(nt);
    std::atomic<bool> ok(true);
    // local levels and level sizes per tile
    parallel_for(nt, [&](int32_t t) {
        int32_t maxl = -1;
        for (int32_t u = cnt[t]; u < cnt[t + 1]; ++u) {
            const int32_t i = rows[u];
            int32_t l = 0;
            for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
                const int32_t j = ci[k];
                if (dep(i, j) && tile_of[j] == t) l = std::max(l, lev[j] + 1);
            }
            lev[i] = l;
            maxl = std::max(maxl, l);
        }
        std::vector<int32_t> &lc = lcount[t];
        lc.assign(maxl + 2, 0);
        for (int32_t u = cnt[t]; u < cnt[t + 1]; ++u) ++lc[lev[rows[u]] + 1];
        int32_t w = 0;
        for (int32_t l = 0; l <= maxl; ++l) w = std::max(w, lc[l + 1]);
        for (int32_t l = 0; l <= maxl; ++l) lc[l + 1] += lc[l];
        nlev_t[t] = maxl + 1;
        width_t[t] = w;
        // local positions (stable by level)
        std::vector<int32_t> f(lc.begin(), lc.end() - 1);
        for (int32_t u = cnt[t]; u < cnt[t + 1]; ++u) {
            const int32_t i = rows[u];
            lpos[i] = f[lev[i]]++;
        }
    });
    h.ntiles = nt;
    h.D = D;
    h.MW = 0;
    h.tlev.assign(nt + 1, 0);
    for (int32_t t = 0; t < nt; ++t) {
        h.tlev[t + 1] = h.tlev[t] + nlev_t[t];
        h.MW = std::max(h.MW, width_t[t]);
        h.maxnl = std::max(h.maxnl, nlev_t[t]);
    }
    if (h.MW > kTileMaxRows || h.MW < 1) return false;
    h.nlev = h.tlev[nt];
    h.lptr.assign((size_t)h.nlev + 1, n);
    const int nslot = D + (fwd ? 0 : 1);
    h.hdr.assign((size_t)n * (1 + D), kTileNone);
    h.kidx.assign((size_t)n * std::max(nslot, 1), -1);
    parallel_for(nt, [&](int32_t t) {
        const std::vector<int32_t> &lc = lcount[t];
        for (int32_t l = 0; l < nlev_t[t]; ++l) h.lptr[h.tlev[t] + l] = cnt[t] + lc[l];
        for (int32_t u = cnt[t]; u < cnt[t + 1]; ++u) {
            const int32_t i = rows[u];
            const size_t p = (size_t)cnt[t] + lpos[i];
            const int32_t lend = lc[lev[i] + 1];   // local position just past row i's level
            h.hdr[p * (1 + D)] = i;
            int d = 0;
            for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
                const int32_t j = ci[k];
                if (!dep(i, j)) continue;
                int32_t code;
                if (tile_of[j] == t && lpos[j] + R >= lend) {
                    code = lpos[j] & (R - 1);
                } else {
                    if (tile_of[j] > t) ok = false;   // the ticket order would not be topological
                    code = -(j + 1);
                }
                h.hdr[p * (1 + D) + 1 + d] = code;
                h.kidx[p * nslot + d] = k;
                ++d;
            }
            if (!fwd) h.kidx[p * nslot + D] = dg[i];
        }
    });
    return ok.load();
}

// modelled time of a sweep with Ty x Tz tiles (us).  The wavefront crosses nx + ny + nz levels in
// all, each at the in-block level time (~0.4 us while a level's rows fit one warp per
// sub-partition, i.e. 32 rows; a tile's blocks beyond 152 run in a second wave), plus ~1.5 us for
// each of the ny/Ty + nz/Tz - 1 hops between blocks.
double tile_model(const int32_t dims[3], int Ty, int Tz) {
    const int nty = (dims[1] + Ty - 1) / Ty, ntz = (dims[2] + Tz - 1) / Tz;
    const int rows = Ty * Tz, waves = (nty * ntz + 151) / 152;
    const double lev_us = 0.4 * std::max(1, (rows + 31) / 32) * waves;
    return 1.5 * (nty + ntz - 1) + lev_us * (dims[0] + dims[1] + dims[2]);
}

}  // namespace

// Natural order on an nx x ny x nz box: the lower dependencies of every row lie at the offsets 1,
// nx and nx*ny (or a subset of them), and n = nx ny nz.  Detected from the host pattern.
static bool tile_grid_find(Ctx *c);

bool tile_grid(Ctx *c) {
    c->tl_dims[0] = c->tl_dims[1] = c->tl_dims[2] = 0;
    if (c->o.ilu_order != CPTR_ILU_NATURAL || c->n_inst > 1) return false;
    IluSym &ys = c->isym;
    if (ys.current && ys.grid >= 0) {   // found for the same pattern at an earlier set-up
        for (int q = 0; q < 3; ++q) c->tl_dims[q] = ys.dims[q];
        return ys.grid == 1;
    }
    const bool found = tile_grid_find(c);
    if (ys.current) {
        ys.grid = found ? 1 : 0;
        for (int q = 0; q < 3; ++q) ys.dims[q] = c->tl_dims[q];
    }
    return found;
}

// the grid dimensions from the pattern's lower offsets (1, nx, nx*ny)
static bool tile_grid_find(Ctx *c) {
    if (host_pattern(c) != CPTR_OK) return false;
    const int32_t n = c->n;
    const std::vector<int32_t> &rp = c->h_rp, &ci = c->h_ci;
    std::vector<int32_t> off;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
            const int32_t o = i - ci[k];
            if (o <= 0) continue;
            if (std::find(off.begin(), off.end(), o) == off.end()) {
                off.push_back(o);
                if (off.size() > 3) return false;
            }
        }
    std::sort(off.begin(), off.end());
    int32_t nx = n, ny = 1, nz = 1;
    if (off.empty()) return false;
    if (off[0] != 1) return false;
    if (off.size() >= 2) {
        nx = off[1];
        if (off.size() == 3) {
            if (off[2] % off[1]) return false;
            ny = off[2] / off[1];
            nz = n / off[2];
        } else {
            ny = n / nx;
        }
    }
    if ((int64_t)nx * ny * nz != n) return false;
    c->tl_dims[0] = nx;
    c->tl_dims[1] = ny;
    c->tl_dims[2] = nz;
    return true;
}

// the k tile shapes of smallest modelled time (tiles of at most kTileMaxRows lines)
void tile_candidates(const Ctx *c, int k, std::vector<std::pair<int, int>> &out) {
    out.clear();
    const int32_t *dims = c->tl_dims;
    if (!dims[0]) return;
    std::vector<std::pair<double, std::pair<int, int>>> all;
    for (int Ty = 1; Ty <= std::min(dims[1], kTileMaxRows); ++Ty)
        for (int Tz = 1; Tz <= std::min(dims[2], kTileMaxRows / Ty); ++Tz)
            all.push_back({tile_model(dims, Ty, Tz), {Ty, Tz}});
    std::sort(all.begin(), all.end());
    for (size_t i = 0; i < all.size() && (int)out.size() < k; ++i) out.push_back(all[i].second);
}

void tile_free(Ctx *c) {
    for (TileTables *t : {&c->tl_f, &c->tl_b}) {
        dfree(t->tlev);
        dfree(t->lptr);
        dfree(t->rec);
        *t = TileTables();
    }
    c->tl_ok = false;
    c->tl_ty = c->tl_tz = 0;
}

cptr_status tile_setup(Ctx *c, int Ty, int Tz) {
    tile_free(c);
    if (!c->tl_dims[0]) return CPTR_OK;
    const int32_t n = c->n, B = c->b, BB = B * B;
    const bool lo = c->o.precision == CPTR_PREC_MIXED;
    const int tsz = lo ? 4 : 8;
    cudaStream_t st = c->stream;
    IluSym &ys = c->isym;
    if (ys.current && ys.tile_ty == Ty && ys.tile_tz == Tz && ys.tile_prec == (int)lo) {
        // the tile structure of the same pattern, from an earlier set-up: copy it, pack the values
        for (int dir = 0; dir < 2; ++dir) {
            const bool fwd = dir == 0;
            TileTables &t = fwd ? c->tl_f : c->tl_b;
            t = ys.tt[dir];
            t.tlev = nullptr;
            t.lptr = nullptr;
            t.rec = nullptr;
            CPTR_TRY(dalloc_t(c, &t.tlev, ys.tlev_n[dir]));
            CPTR_TRY(dalloc_t(c, &t.lptr, ys.lptr_n[dir]));
            CPTR_CUDA_TRY(c, cudaMemcpyAsync(t.tlev, ys.tt[dir].tlev, sizeof(int32_t) * ys.tlev_n[dir],
                                             cudaMemcpyDeviceToDevice, st));
            CPTR_CUDA_TRY(c, cudaMemcpyAsync(t.lptr, ys.tt[dir].lptr, sizeof(int32_t) * ys.lptr_n[dir],
                                             cudaMemcpyDeviceToDevice, st));
            CPTR_TRY(dalloc(c, reinterpret_cast<void **>(&t.rec), (size_t)n * t.RS));
            const int nslot = t.D + (fwd ? 0 : 1);
            const int H = hdr_bytes(t.D);
            if (lo)
                (k_tile_pack<float><<<nblk(n, 256), 256, 0, st>>>(n, t.D, BB, t.RS, H, nslot, ys.hdr[dir], ys.kidx[dir],
                                                                   c->LU, t.rec), note_launch());
            else
                (k_tile_pack<double><<<nblk(n, 256), 256, 0, st>>>(n, t.D, BB, t.RS, H, nslot, ys.hdr[dir], ys.kidx[dir],
                                                                    c->LU, t.rec), note_launch());
            CPTR_CUDA_TRY(c, cudaGetLastError());
        }
        c->tl_ok = true;
        c->tl_ty = Ty;
        c->tl_tz = Tz;
        return CPTR_OK;
    }
    CPTR_TRY(host_pattern(c));
    // the structure built here replaces the kept one (if this set-up's pattern is the kept one)
    const bool keep = ys.current;
    if (keep) {
        for (int dir = 0; dir < 2; ++dir) {
            dfree(ys.tt[dir].tlev); dfree(ys.tt[dir].lptr); dfree(ys.hdr[dir]); dfree(ys.kidx[dir]);
            ys.tt[dir] = TileTables();
            ys.hdr[dir] = ys.kidx[dir] = nullptr;
        }
        ys.tile_ty = ys.tile_tz = 0;
        ys.tile_prec = -1;
    }
    for (int dir = 0; dir < 2; ++dir) {
        const bool fwd = dir == 0;
        TileHost h;
        // the ring holds the last R solved rows of a tile; 4 levels of the widest tile at least
        int R = 256;
        while (R < 4 * Ty * Tz) R *= 2;
        if (!tile_build(n, c->h_rp, c->h_ci, c->h_diag, c->tl_dims, Ty, Tz, fwd, R, h)) {
            tile_free(c);
            return CPTR_OK;
        }
        TileTables &t = fwd ? c->tl_f : c->tl_b;
        t.ntiles = h.ntiles;
        t.nlev = h.nlev;
        t.D = h.D;
        t.MW = h.MW;
        t.R = R;
        t.maxnl = h.maxnl;
        t.RS = rec_bytes(h.D, BB, tsz, fwd);
        const int ssz = fwd ? 8 : tsz;   // right-hand side: r (FP64, or FP32 in the FP32 stage) or y
        size_t smem = 0;
        // the deepest pipeline that fits (P levels of lookahead for the values, 2P for the records)
        int P = 0;
        for (int p : {4, 2, 1}) {
            smem = kTileBar + lv_bytes(h.maxnl) + (size_t)(2 * p + 1) * t.MW * t.RS + (size_t)(p + 1) * t.MW * val_bytes(h.D, B, ssz) +
                   (size_t)R * B * tsz;
            if (smem <= kTileSmemMax) {
                P = p;
                break;
            }
        }
        if (P < 1) {
            tile_free(c);
            return CPTR_OK;
        }
        t.P = P;
        t.smem = (int32_t)smem;
        t.threads = ((4 * t.MW + 31) / 32) * 32 + 32;   // consumer warps and one producer warp
        t.grid = std::min(h.ntiles, 152);
        CPTR_TRY(dalloc_t(c, &t.tlev, h.tlev.size()));
        CPTR_TRY(dalloc_t(c, &t.lptr, h.lptr.size()));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(t.tlev, h.tlev.data(), sizeof(int32_t) * h.tlev.size(), cudaMemcpyHostToDevice, st));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(t.lptr, h.lptr.data(), sizeof(int32_t) * h.lptr.size(), cudaMemcpyHostToDevice, st));
        int32_t *dh = nullptr, *dk = nullptr;
        CPTR_TRY(dalloc_t(c, &dh, h.hdr.size()));
        CPTR_TRY(dalloc_t(c, &dk, h.kidx.size()));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(dh, h.hdr.data(), sizeof(int32_t) * h.hdr.size(), cudaMemcpyHostToDevice, st));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(dk, h.kidx.data(), sizeof(int32_t) * h.kidx.size(), cudaMemcpyHostToDevice, st));
        CPTR_TRY(dalloc(c, reinterpret_cast<void **>(&t.rec), (size_t)n * t.RS));
        const int nslot = h.D + (fwd ? 0 : 1);
        const int H = hdr_bytes(h.D);
        if (lo)
            (k_tile_pack<float><<<nblk(n, 256), 256, 0, st>>>(n, h.D, BB, t.RS, H, nslot, dh, dk, c->LU, t.rec), note_launch());
        else
            (k_tile_pack<double><<<nblk(n, 256), 256, 0, st>>>(n, h.D, BB, t.RS, H, nslot, dh, dk, c->LU, t.rec), note_launch());
        CPTR_CUDA_TRY(c, cudaGetLastError());
        CPTR_CUDA_TRY(c, cudaStreamSynchronize(st));   // the host tables are freed on return
        if (keep) {   // kept for the next set-up of this pattern: sizes, level tables, headers, indices
            ys.tt[dir] = t;
            ys.tt[dir].rec = nullptr;
            ys.tt[dir].tlev = ys.tt[dir].lptr = nullptr;
            ys.tlev_n[dir] = h.tlev.size();
            ys.lptr_n[dir] = h.lptr.size();
            CPTR_TRY(dalloc_t(c, &ys.tt[dir].tlev, h.tlev.size()));
            CPTR_TRY(dalloc_t(c, &ys.tt[dir].lptr, h.lptr.size()));
            CPTR_CUDA_TRY(c, cudaMemcpyAsync(ys.tt[dir].tlev, t.tlev, sizeof(int32_t) * h.tlev.size(),
                                             cudaMemcpyDeviceToDevice, st));
            CPTR_CUDA_TRY(c, cudaMemcpyAsync(ys.tt[dir].lptr, t.lptr, sizeof(int32_t) * h.lptr.size(),
                                             cudaMemcpyDeviceToDevice, st));
            ys.hdr[dir] = dh;
            ys.kidx[dir] = dk;
        } else {
            dfree(dh);
            dfree(dk);
        }
    }
    if (keep) {
        ys.tile_ty = Ty;
        ys.tile_tz = Tz;
        ys.tile_prec = (int)lo;
    }
    c->tl_ok = true;
    c->tl_ty = Ty;
    c->tl_tz = Tz;
    return CPTR_OK;
}

namespace {
template <int B, typename T, typename ST, typename XT, bool FWD>
void tile_launch(const Ctx *c, const TileTables &t, const ST *src, T *vec, double *out, const XT *dp, const XT *dT,
                 const double *never) {
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmemMax);
        (kern<<<t.grid, t.threads, t.smem, c->stream>>>(t.ntiles, t.tlev, t.lptr, t.rec, t.RS, t.D, t.R, t.MW, t.maxnl, src, vec,
                                                       out, c->ps, c->ts, dp, dT, c->sf_ticket, c->ks, never,
                                                       c->sf_sleep),
         note_launch());
    };
    if (t.P == 4) go(k_ilu_tile<B, T, ST, XT, FWD, 4>);
    else if (t.P == 2) go(k_ilu_tile<B, T, ST, XT, FWD, 2>);
    else go(k_ilu_tile<B, T, ST, XT, FWD, 1>);
}

template <int B, typename T, typename RT, typename XT>
void tile_apply_b(const Ctx *c, const RT *r, double *z, const XT *dp, const XT *dT) {
    T *y = (T *)c->sf_y, *zz = (T *)c->sf_z;
    int pf = prof_begin(c, PF_ILU_FWD);
    tile_launch<B, T, RT, XT, true>(c, c->tl_f, r, y, nullptr, (const XT *)nullptr, (const XT *)nullptr,
                                    c->inject_wait ? c->never : nullptr);
    prof_end(c, pf);
    pf = prof_begin(c, PF_ILU_BWD);
    tile_launch<B, T, T, XT, false>(c, c->tl_b, y, zz, z, dp, dT, nullptr);
    prof_end(c, pf);
}
}  // namespace

template <typename T, typename RT, typename XT>
void tile_apply(const Ctx *c, const RT *r, double *z, const XT *dp, const XT *dT) {
    if (c->b == 3) tile_apply_b<3, T, RT, XT>(c, r, z, dp, dT);
    else tile_apply_b<4, T, RT, XT>(c, r, z, dp, dT);
}
template void tile_apply<double, double, double>(const Ctx *, const double *, double *, const double *, const double *);
template void tile_apply<float, double, double>(const Ctx *, const double *, double *, const double *, const double *);
template void tile_apply<float, float, float>(const Ctx *, const float *, double *, const float *, const float *);

}  // namespace cptr
