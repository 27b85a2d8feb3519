// Sparse building blocks of the CPTR solve: BSR SpMV with b x b register blocks, the decoupling
// A' = W A (Sec. 2.2.2 eq. weighted, Sec. 3.5 eq. scaling), the extraction of the scalar p-T
// blocks on the cell pattern (Sec. 3.2 eq. A00), the stage-1 residual v - A' R_0^T x_0
// (Sec. 3 "Two-stage preconditioners", step 2), scalar CSR SpMV, and a device prefix scan.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <vector>

#include <mutex>

#include "common.cuh"

namespace cptr {

static std::atomic<int64_t> g_launches{0};
static thread_local bool t_capturing = false;
static thread_local int64_t t_captured = 0;
void note_launch() {
    if (t_capturing) ++t_captured;
    else g_launches.fetch_add(1, std::memory_order_relaxed);
}
void note_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
void begin_capture_count() { t_capturing = true; t_captured = 0; }
int64_t end_capture_count() { t_capturing = false; return t_captured; }

double host_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
void setup_tick(Ctx *c, int phase, double *t0) {
    cudaStreamSynchronize(c->stream);
    double t = host_ms();
    c->prof.setup_ms[phase] += t - *t0;
    *t0 = t;
}

int prof_begin(const Ctx *c, int fam) {
    Prof &p = c->prof;
    if (!(p.mask & (1u << (fam < PF_FAMILIES ? fam : 7)))) return -1;
    if (2 * (p.used + 1) > p.ev.size()) {
        for (int k = 0; k < 64; ++k) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return -1;
            p.ev.push_back(e);
        }
        p.fam.resize(p.ev.size() / 2);
    }
    size_t s = p.used++;
    p.fam[s] = fam;
    if (p.capturing) {
        // inside stream capture a plain record is only a capture dependency: ask for a graph node
        p.gslots.push_back(s);
        cudaEventRecordWithFlags(p.ev[2 * s], c->stream, cudaEventRecordExternal);
    } else {
        cudaEventRecord(p.ev[2 * s], c->stream);
    }
    return (int)s;
}
void prof_begin_capture(Ctx *c) {
    c->prof.capturing = true;
    c->prof.gslots.clear();
}
void prof_end_capture(Ctx *c) {
    // the captured slots stay reserved at the front of the pool; direct launches use the rest
    c->prof.capturing = false;
}
cptr_status prof_collect_graph(Ctx *c) {
    Prof &p = c->prof;
    for (size_t s : p.gslots) {
        float ms = 0.f;
        CPTR_CUDA_TRY(c, cudaEventElapsedTime(&ms, p.ev[2 * s], p.ev[2 * s + 1]));
        p.ms[p.fam[s]] += ms;
        p.cnt[p.fam[s]] += 1;
    }
    return CPTR_OK;
}
void prof_end(const Ctx *c, int slot) {
    if (slot < 0) return;
    if (c->prof.capturing) cudaEventRecordWithFlags(c->prof.ev[2 * (size_t)slot + 1], c->stream, cudaEventRecordExternal);
    else cudaEventRecord(c->prof.ev[2 * (size_t)slot + 1], c->stream);
}
void prof_reset(Ctx *c) {
    c->prof.used = c->prof.gslots.empty() ? 0 : c->prof.gslots.back() + 1;
    for (int f = 0; f < PF_N; ++f) { c->prof.ms[f] = 0.0; c->prof.cnt[f] = 0; }
}
cptr_status prof_collect(Ctx *c) {
    Prof &p = c->prof;
    size_t first = p.gslots.empty() ? 0 : p.gslots.back() + 1;
    for (size_t s = first; s < p.used; ++s) {
        float ms = 0.f;
        CPTR_CUDA_TRY(c, cudaEventSynchronize(p.ev[2 * s + 1]));
        CPTR_CUDA_TRY(c, cudaEventElapsedTime(&ms, p.ev[2 * s], p.ev[2 * s + 1]));
        p.ms[p.fam[s]] += ms;
        p.cnt[p.fam[s]] += 1;
    }
    p.used = first;
    return CPTR_OK;
}

#ifdef CPTR_CHECK
namespace {
struct CheckFns {
    cudaError_t (*fetch)(CheckRec *);
    cudaError_t (*clear)();
};
std::vector<CheckFns> &check_list() {
    static std::vector<CheckFns> v;   // filled by static initialisers at load time
    return v;
}
std::mutex g_check_mu;
const char *check_site(int s) {
    switch (s) {
    case CHK_SELL_COL: return "SELL SpMV column";
    case CHK_CSR_COL: return "CSR SpMV column";
    case CHK_VC_COL: return "V-cycle column";
    case CHK_ILU_DEP: return "ILU sweep dependency";
    case CHK_ILU_PAIR: return "paired-level term";
    case CHK_FACTOR_COL: return "ILU factorisation column";
    case CHK_FACTOR_DEP: return "ILU factorisation pivot position";
    default: return "index";
    }
}
}  // namespace
void check_register(cudaError_t (*fetch)(CheckRec *), cudaError_t (*clear)()) {
    std::lock_guard<std::mutex> lock(g_check_mu);
    check_list().push_back({fetch, clear});
}
cptr_status check_report(Ctx *c) {
    std::lock_guard<std::mutex> lock(g_check_mu);
    CPTR_CUDA_TRY(c, cudaDeviceSynchronize());
    CheckRec first{};
    int64_t total = 0;
    for (const CheckFns &f : check_list()) {
        CheckRec r{};
        CPTR_CUDA_TRY(c, f.fetch(&r));
        if (r.count > 0) {
            if (total == 0) first = r;
            total += r.count;
            CPTR_CUDA_TRY(c, f.clear());
        }
    }
    if (total == 0) return CPTR_OK;
    return c->fail(CPTR_ECHECK, std::string("index check failed: ") + check_site(first.site) + " " +
                                    std::to_string(first.index) + " outside [0, " + std::to_string(first.bound) +
                                    ") (" + std::to_string(total) + " failed accesses skipped)");
}
#else
cptr_status check_report(Ctx *) { return CPTR_OK; }
#endif

static thread_local Ctx *t_scope = nullptr;
CtxScope::CtxScope(Ctx *c) : prev(t_scope) { t_scope = c; }
CtxScope::~CtxScope() { t_scope = prev; }

cptr_status dalloc(Ctx *c, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = c->pool ? cudaMallocFromPoolAsync(p, bytes, c->pool, c->stream) : cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return c->fail(CPTR_ENOMEM, std::string("device allocation of ") + std::to_string(bytes) + " bytes: " +
                                        cudaGetErrorString(e));
    }
    return CPTR_OK;
}
void dfree(void *p) {
    if (!p) return;
    if (t_scope && t_scope->pool) cudaFreeAsync(p, t_scope->stream);
    else cudaFree(p);
}
cptr_status copy_to_host(Ctx *c, void *dst, const void *src, size_t bytes) {
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream));
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return CPTR_OK;
}
void csr_free(Csr &a) {
    dfree(a.rp); dfree(a.ci); dfree(a.v);
    a = Csr{};
}

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ------------------------------------------------------------------------------------------------
// exclusive prefix scan of int32: tiles of 2048 (256 threads x 8 items)
constexpr int kScanT = 256, kScanI = 8, kScanTile = kScanT * kScanI;

__device__ __forceinline__ int32_t block_scan_excl(int32_t v, int32_t *total) {
    __shared__ int32_t warp_sum[kScanT / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int32_t s = lane < kScanT / 32 ? warp_sum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kScanT / 32) warp_sum[lane] = s;
    }
    __syncthreads();
    int32_t before = (wid > 0 ? warp_sum[wid - 1] : 0) + x - v;
    *total = warp_sum[kScanT / 32 - 1];
    __syncthreads();
    return before;
}

__global__ void k_tile_sum(const int32_t *in, int32_t n, int32_t *tsum) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanI;
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanI; ++k)
        if (base + k < n) s += in[base + k];
    int32_t tot;
    block_scan_excl(s, &tot);
    if (threadIdx.x == 0) tsum[blockIdx.x] = tot;
}

__global__ void k_tile_scan(const int32_t *in, int32_t n, const int32_t *toff, int32_t *out) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanI;
    int32_t loc[kScanI];
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanI; ++k) {
        loc[k] = (base + k < n) ? in[base + k] : 0;
        s += loc[k];
    }
    int32_t tot;
    int32_t run = block_scan_excl(s, &tot) + (toff ? toff[blockIdx.x] : 0);
#pragma unroll
    for (int k = 0; k < kScanI; ++k) {
        if (base + k < n) out[base + k] = run;
        run += loc[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanT - 1) out[n] = run;
}

// out[0..n] = exclusive scan of in[0..n-1], out[n] = total.  out may not alias in.
static cptr_status scan_rec(Ctx *c, const int32_t *in, int32_t *out, int32_t n, int32_t *tmp) {
    if (n <= 0) {
        CPTR_CUDA_TRY(c, cudaMemsetAsync(out, 0, sizeof(int32_t), c->stream));
        return CPTR_OK;
    }
    int32_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        (k_tile_scan<<<1, kScanT, 0, c->stream>>>(in, n, nullptr, out), note_launch());
        return CPTR_OK;
    }
    int32_t *tsum = tmp, *toff = tmp + tiles;
    (k_tile_sum<<<tiles, kScanT, 0, c->stream>>>(in, n, tsum), note_launch());
    CPTR_TRY(scan_rec(c, tsum, toff, tiles, tmp + 2 * tiles + 1));
    (k_tile_scan<<<tiles, kScanT, 0, c->stream>>>(in, n, toff, out), note_launch());
    return CPTR_OK;
}

cptr_status scan_exclusive(Ctx *c, const int32_t *in, int32_t *out, int32_t n, int32_t *total_host) {
    int64_t need = 4 * ((int64_t)n / kScanTile + 8) + 64;
    if (need > c->scan_tmp_len) {
        dfree(c->scan_tmp);
        c->scan_tmp = nullptr;
        CPTR_TRY(dalloc_t(c, &c->scan_tmp, (size_t)need));
        c->scan_tmp_len = need;
    }
    CPTR_TRY(scan_rec(c, in, out, n, c->scan_tmp));
    CPTR_CUDA_TRY(c, cudaGetLastError());
    if (total_host) {
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(total_host, out + n, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    return CPTR_OK;
}

// ------------------------------------------------------------------------------------------------
// decoupling: block row i of A' = W_i * (block row i of A); each entry is the sum over the slot
// index of separately rounded products, in slot order, so that A' is reproducible bit for bit
template <int B>
__global__ void k_decouple(int32_t n, const int32_t *rp, const double *Araw, const double *W, double *A) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double w[B * B];
#pragma unroll
    for (int t = 0; t < B * B; ++t) w[t] = W ? W[(int64_t)i * B * B + t] : ((t / B == t % B) ? 1.0 : 0.0);
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
        const double *a = Araw + (int64_t)k * B * B;
        double in[B * B];
#pragma unroll
        for (int t = 0; t < B * B; ++t) in[t] = a[t];
#pragma unroll
        for (int r = 0; r < B; ++r)
#pragma unroll
            for (int cc = 0; cc < B; ++cc) {
                double s = 0.0;
#pragma unroll
                for (int q = 0; q < B; ++q) s = __dadd_rn(s, __dmul_rn(w[r * B + q], in[q * B + cc]));
                A[(int64_t)k * B * B + r * B + cc] = s;
            }
    }
}

void launch_decouple(const Ctx *c, const double *Araw, const double *W, double *A) {
    if (c->b == 3) (k_decouple<3><<<nblk(c->n, 128), 128, 0, c->stream>>>(c->n, c->rp, Araw, W, A), note_launch());
    else (k_decouple<4><<<nblk(c->n, 128), 128, 0, c->stream>>>(c->n, c->rp, Araw, W, A), note_launch());
}

template <int B>
__global__ void k_weight_vec(int32_t n, const double *W, const double *rhs, double *out) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v[B];
#pragma unroll
    for (int q = 0; q < B; ++q) v[q] = rhs[(int64_t)i * B + q];
#pragma unroll
    for (int r = 0; r < B; ++r) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < B; ++q) s = __dadd_rn(s, __dmul_rn(W ? W[(int64_t)i * B * B + r * B + q] : (r == q ? 1.0 : 0.0), v[q]));
        out[(int64_t)i * B + r] = s;
    }
}

void launch_weight_vec(const Ctx *c, const double *W, const double *rhs, double *out) {
    if (c->b == 3) (k_weight_vec<3><<<nblk(c->n, 256), 256, 0, c->stream>>>(c->n, W, rhs, out), note_launch());
    else (k_weight_vec<4><<<nblk(c->n, 256), 256, 0, c->stream>>>(c->n, W, rhs, out), note_launch());
}

// scalar field (u, w) of every block: out[k] = A'[k](u, w)
__global__ void k_extract(int32_t nnzb, int b, const double *A, int u, int w, double *out) {
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nnzb) out[k] = A[(int64_t)k * b * b + u * b + w];
}
// field (u, w) of G A' for a primary slot u (decoupling row ru of D): a(i,u; j,w) - sum over the slots
// s ascending with D_i[ru][s] != 0 of D_i[ru][s] a(i,s; j,w), products and differences rounded apart
__global__ void k_extract_g(int32_t n, int b, const int32_t *rp, const double *A, int u, int w, int ru,
                            const double *D, double *out) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *Di = D + ((int64_t)i * 2 + ru) * b;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
        const double *blk = A + (int64_t)k * b * b;
        double v = blk[u * b + w];
        for (int s = 0; s < b; ++s)
            if (Di[s] != 0.0) v = __dsub_rn(v, __dmul_rn(Di[s], blk[s * b + w]));
        out[k] = v;
    }
}
void launch_extract(const Ctx *c, int u, int w, double *out) {
    const bool prim = u == c->ps || (u == c->ts && c->o.stage1 != CPTR_STAGE1_CPR);
    if (c->Ddec && prim)
        (k_extract_g<<<nblk(c->n, 256), 256, 0, c->stream>>>(c->n, c->b, c->rp, c->A, u, w, u == c->ps ? 0 : 1,
                                                             c->Ddec, out), note_launch());
    else
        (k_extract<<<nblk(c->nnzb, 256), 256, 0, c->stream>>>(c->nnzb, c->b, c->A, u, w, out), note_launch());
}

// D_i = X_i Y_i^{-1} of the decoupling operator (see cptr_options.decouple): X_i (primary rows x
// secondary columns) and Y_i (secondary x secondary) from the cell's diagonal block (QI) or summed
// over the blocks (j, i) of its block column, rows j ascending (TI; block (j, i) found by binary
// search in row j, flag 1 if missing); Y_i^{-1} by Gauss-Jordan with partial pivoting (flag 2 if
// singular); D = X Y^{-1} summed over u ascending.  Every operation separately rounded.
__global__ void k_decoupling(int32_t n, int b, int ps, int ts, int nprim, int kind, const int32_t *rp,
                             const int32_t *ci, const double *A, double *D, int32_t *flag) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int prim[2] = {ps, ts}, sec[4], ns = 0;
    for (int q = 0; q < b; ++q) {
        bool p = q == ps || (nprim == 2 && q == ts);
        if (!p) sec[ns++] = q;
    }
    double X[2][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}}, a[3][6];
    double Y[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
        const int32_t j = ci[k];
        int32_t kk = -1;
        if (kind == CPTR_DECOUPLE_QI) {
            if (j != i) continue;
            kk = k;
        } else {
            int32_t lo = rp[j], hi = rp[j + 1] - 1;
            while (lo <= hi) {
                const int32_t mid = (lo + hi) >> 1;
                if (ci[mid] == i) { kk = mid; break; }
                if (ci[mid] < i) lo = mid + 1;
                else hi = mid - 1;
            }
            if (kk < 0) { atomicExch(flag, 1); return; }
        }
        const double *blk = A + (int64_t)kk * b * b;
        for (int r = 0; r < nprim; ++r)
            for (int t = 0; t < ns; ++t) X[r][t] = __dadd_rn(X[r][t], blk[prim[r] * b + sec[t]]);
        for (int r = 0; r < ns; ++r)
            for (int t = 0; t < ns; ++t) Y[r][t] = __dadd_rn(Y[r][t], blk[sec[r] * b + sec[t]]);
        if (kind == CPTR_DECOUPLE_QI) break;
    }
    for (int r = 0; r < ns; ++r)
        for (int q = 0; q < 2 * ns; ++q) a[r][q] = q < ns ? Y[r][q] : (q - ns == r ? 1.0 : 0.0);
    for (int k = 0; k < ns; ++k) {
        int p = k;
        for (int r = k + 1; r < ns; ++r)
            if (fabs(a[r][k]) > fabs(a[p][k])) p = r;
        if (a[p][k] == 0.0) { atomicExch(flag, 2); return; }
        if (p != k)
            for (int q = 0; q < 2 * ns; ++q) { const double t = a[k][q]; a[k][q] = a[p][q]; a[p][q] = t; }
        const double inv = __ddiv_rn(1.0, a[k][k]);
        for (int q = 0; q < 2 * ns; ++q) a[k][q] = __dmul_rn(a[k][q], inv);
        for (int r = 0; r < ns; ++r) {
            if (r == k) continue;
            const double f = a[r][k];
            for (int q = 0; q < 2 * ns; ++q) a[r][q] = __dsub_rn(a[r][q], __dmul_rn(f, a[k][q]));
        }
    }
    double *Di = D + (int64_t)i * 2 * b;
    for (int q = 0; q < 2 * b; ++q) Di[q] = 0.0;
    for (int r = 0; r < nprim; ++r)
        for (int t = 0; t < ns; ++t) {
            double d = 0.0;
            for (int u = 0; u < ns; ++u) d = __dadd_rn(d, __dmul_rn(X[r][u], a[u][ns + t]));
            Di[r * b + sec[t]] = d;
        }
}

cptr_status decoupling_setup(Ctx *c) {
    CPTR_TRY(dalloc_t(c, &c->Ddec, (size_t)c->n * 2 * c->b));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(c->flag, 0, sizeof(int32_t), c->stream));
    const int nprim = c->o.stage1 == CPTR_STAGE1_CPR ? 1 : 2;
    (k_decoupling<<<nblk(c->n, 128), 128, 0, c->stream>>>(c->n, c->b, c->ps, c->ts, nprim, c->o.decouple, c->rp,
                                                         c->ci, c->A, c->Ddec, c->flag), note_launch());
    CPTR_CUDA_TRY(c, cudaGetLastError());
    int32_t f = 0;
    CPTR_TRY(copy_to_host(c, &f, c->flag, sizeof(int32_t)));
    if (f == 1) return c->fail(CPTR_EINVAL, "True-IMPES decoupling needs a structurally symmetric pattern");
    if (f == 2) return c->fail(CPTR_ESINGULAR, "decoupling: singular secondary block");
    return CPTR_OK;
}

__global__ void k_check_finite(const double *v, int64_t n, int32_t *flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int bad = 0;
    for (; i < n; i += stride) bad |= !isfinite(v[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}
void launch_check_finite(const Ctx *c, const double *v, int64_t n, int32_t *flag) {
    (k_check_finite<<<4 * 152, 256, 0, c->stream>>>(v, n, flag), note_launch());
}

// ------------------------------------------------------------------------------------------------
// A' is kept for the solve in a sliced-ELL block layout (SELL-32): block rows are grouped in
// chunks of 32; chunk c holds w_c block slots per row (its longest row; shorter rows are padded
// with zero blocks pointing at column 0) stored slot-major and lane-minor, so that the 32 rows
// of a chunk read each block entry with one fully coalesced 256-byte access:
//   col[(off_c + s) * 32 + lane],  val[((off_c + s) * b*b + e) * 32 + lane]
// One thread computes one block row.
cptr_status sell_build(Ctx *c) {
    const int32_t n = c->n, B = c->b, nch = (n + 31) / 32;
    std::vector<int64_t> off(nch + 1, 0);
    std::vector<int32_t> w(nch, 0);
    for (int32_t ch = 0; ch < nch; ++ch) {
        int32_t mx = 0;
        for (int32_t r = ch * 32; r < std::min(n, ch * 32 + 32); ++r) mx = std::max(mx, c->h_rp[r + 1] - c->h_rp[r]);
        w[ch] = mx;
        off[ch + 1] = off[ch] + mx;
    }
    c->sell_nch = nch;
    const int64_t slots = off[nch] * 32;
    CPTR_TRY(dalloc_t(c, &c->sell_off, (size_t)nch + 1));
    CPTR_TRY(dalloc_t(c, &c->sell_col, (size_t)slots));
    CPTR_TRY(dalloc_t(c, &c->sell_val, (size_t)slots * B * B));
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->sell_off, off.data(), sizeof(int64_t) * (nch + 1), cudaMemcpyHostToDevice, c->stream));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(c->sell_col, 0, sizeof(int32_t) * slots, c->stream));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(c->sell_val, 0, sizeof(double) * slots * B * B, c->stream));
    launch_bsr_to_sell(c);
    CPTR_CUDA_TRY(c, cudaGetLastError());
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->sell_bytes = slots * (4 + 8 * B * B) + (nch + 1) * 8;
    c->sell_nvals = slots * B * B;
    return CPTR_OK;
}

__global__ void k_bsr_to_sell(int32_t n, int B, const int32_t *rp, const int32_t *ci, const double *A,
                              const int64_t *off, int32_t *col, double *val) {
    int32_t row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    int32_t ch = row >> 5, lane = row & 31;
    int64_t o = off[ch];
    for (int32_t k = rp[row]; k < rp[row + 1]; ++k) {
        int64_t slot = o + (k - rp[row]);
        col[slot * 32 + lane] = ci[k];
        for (int e = 0; e < B * B; ++e) val[(slot * B * B + e) * 32 + lane] = A[(int64_t)k * B * B + e];
    }
}
void launch_bsr_to_sell(const Ctx *c) {
    (k_bsr_to_sell<<<nblk(c->n, 256), 256, 0, c->stream>>>(c->n, c->b, c->rp, c->ci, c->A, c->sell_off, c->sell_col,
                                                            c->sell_val), note_launch());
}

// MODE 0: y = A' x;  MODE 1: y = v - A' x;  MODE 2: y = v - A' R_0^T [dp; dT] (only the p and T
// columns of each block are read; dT may be null for CPR)
template <int B, int MODE>
__global__ void __launch_bounds__(512) k_sell_spmv(int32_t n, const int64_t *__restrict__ off,
                                                    const int32_t *__restrict__ col, const double *__restrict__ val,
                                                    const double *__restrict__ x, const double *__restrict__ v,
                                                    double *__restrict__ y, int ps, int ts,
                                                    const double *__restrict__ dp, const double *__restrict__ dT) {
    int32_t row = blockIdx.x * blockDim.x + threadIdx.x;
    int32_t ch = row >> 5, lane = row & 31;
    if (row >= ((n + 31) & ~31)) return;
    const int64_t o0 = __ldg(off + ch), o1 = __ldg(off + ch + 1);
    double acc[B];
#pragma unroll
    for (int r = 0; r < B; ++r) acc[r] = 0.0;
    for (int64_t sl = o0; sl < o1; ++sl) {
        const int32_t cidx = (int32_t)chk(__ldg(col + sl * 32 + lane), n, CHK_SELL_COL);
        const double *a = val + sl * B * B * 32 + lane;
        if (MODE == 2) {
            const double xp = __ldg(dp + cidx);
            const double xt = dT ? __ldg(dT + cidx) : 0.0;
#pragma unroll
            for (int r = 0; r < B; ++r) {
                acc[r] = fma(__ldg(a + (r * B + ps) * 32), xp, acc[r]);
                if (dT) acc[r] = fma(__ldg(a + (r * B + ts) * 32), xt, acc[r]);
            }
        } else {
            double xv[B];
#pragma unroll
            for (int q = 0; q < B; ++q) xv[q] = __ldg(x + (int64_t)cidx * B + q);
#pragma unroll
            for (int r = 0; r < B; ++r)
#pragma unroll
                for (int q = 0; q < B; ++q) acc[r] = fma(__ldg(a + (r * B + q) * 32), xv[q], acc[r]);
        }
    }
    if (row < n) {
#pragma unroll
        for (int r = 0; r < B; ++r) {
            int64_t oo = (int64_t)row * B + r;
            y[oo] = MODE == 0 ? acc[r] : v[oo] - acc[r];
        }
    }
}

template <int MODE>
static void sell_dispatch(const Ctx *c, const double *x, const double *v, double *y, const double *dp,
                          const double *dT) {
    const int T = c->sell_shape.T;
    unsigned grid = nblk((int64_t)c->sell_nch * 32, T);
    if (c->b == 3)
        (k_sell_spmv<3, MODE><<<grid, T, 0, c->stream>>>(c->n, c->sell_off, c->sell_col, c->sell_val, x, v, y, c->ps,
                                                         c->ts, dp, dT), note_launch());
    else
        (k_sell_spmv<4, MODE><<<grid, T, 0, c->stream>>>(c->n, c->sell_off, c->sell_col, c->sell_val, x, v, y, c->ps,
                                                         c->ts, dp, dT), note_launch());
}
void launch_bsr_spmv(const Ctx *c, const double *x, double *y) { sell_dispatch<0>(c, x, nullptr, y, nullptr, nullptr); }
void launch_bsr_resid(const Ctx *c, const double *x, const double *v, double *y) {
    sell_dispatch<1>(c, x, v, y, nullptr, nullptr);
}
void launch_bsr_resid_pt(const Ctx *c, const double *dp, const double *dT, const double *v, double *b1) {
    sell_dispatch<2>(c, nullptr, v, b1, dp, dT);
}

// ------------------------------------------------------------------------------------------------
// scalar CSR SpMV with G lanes per row, values VT (double, float or bf16), vectors and sums XT:
// mode 0 y = A x, mode 1 y = c0 - A x, mode 2 y += A x
__device__ __forceinline__ double val_ld(const double *p) { return __ldg(p); }
__device__ __forceinline__ float val_ld(const float *p) { return __ldg(p); }
__device__ __forceinline__ float val_ld(const bf16 *p) {
    return __bfloat162float(__ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short *>(p))));
}

template <int G, typename VT, typename XT>
__global__ void __launch_bounds__(512) k_csr_spmv(int32_t n, const int32_t *__restrict__ rp,
                                                   const int32_t *__restrict__ ci, const VT *__restrict__ v,
                                                   const XT *__restrict__ x, XT *__restrict__ y, int mode,
                                                   const XT *__restrict__ c0, int32_t ncol, const XT *__restrict__ ts,
                                                   XT *__restrict__ to) {
    pdl_wait();
    int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t row = (int32_t)(gid / G);
    int lane = threadIdx.x % G;
    XT acc = 0;
    if (row < n) {
        int32_t k1 = __ldg(rp + row + 1);
        if (G == 1) {
            acc = row_dot_batched<4>(__ldg(rp + row), k1, ci, [&](int32_t k) { return (XT)val_ld(v + k); },
                                     [&](int32_t j) { return __ldg(x + chk(j, ncol, CHK_CSR_COL)); }, acc);
        } else {
            for (int32_t k = __ldg(rp + row) + lane; k < k1; k += G)
                acc = fma((XT)val_ld(v + k), __ldg(x + chk(__ldg(ci + k), ncol, CHK_CSR_COL)), acc);
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, G);
    if (row < n && lane == 0) {
        if (mode == 0) y[row] = acc;
        else if (mode == 1) y[row] = c0[row] - acc;
        else y[row] += acc;
        // the output feeds a V-cycle level: its first smoothing step t = D^{-1} y as well
        if (to) to[row] = ts[row] * (mode == 0 ? acc : c0[row] - acc);
    }
}

template <typename VT, typename XT>
void launch_csr_spmv_t(cudaStream_t s, int32_t n, int32_t nnz, const int32_t *rp, const int32_t *ci, const VT *v,
                       const XT *x, XT *y, int mode, const XT *c0, Shape sh, int32_t ncol, const XT *ts, XT *to) {
    const int G = sh.G ? sh.G : lanes_for(n, nnz), T = sh.T;
    unsigned grid = nblk((int64_t)n * G, T);
    switch (G) {
    case 1: launch_pdl(k_csr_spmv<1, VT, XT>, grid, T, 0, s, n, rp, ci, v, x, y, mode, c0, ncol, ts, to); break;
    case 2: launch_pdl(k_csr_spmv<2, VT, XT>, grid, T, 0, s, n, rp, ci, v, x, y, mode, c0, ncol, ts, to); break;
    case 4: launch_pdl(k_csr_spmv<4, VT, XT>, grid, T, 0, s, n, rp, ci, v, x, y, mode, c0, ncol, ts, to); break;
    case 8: launch_pdl(k_csr_spmv<8, VT, XT>, grid, T, 0, s, n, rp, ci, v, x, y, mode, c0, ncol, ts, to); break;
    case 16: launch_pdl(k_csr_spmv<16, VT, XT>, grid, T, 0, s, n, rp, ci, v, x, y, mode, c0, ncol, ts, to); break;
    default: launch_pdl(k_csr_spmv<32, VT, XT>, grid, T, 0, s, n, rp, ci, v, x, y, mode, c0, ncol, ts, to); break;
    }
}
template void launch_csr_spmv_t<double, double>(cudaStream_t, int32_t, int32_t, const int32_t *, const int32_t *,
                                                const double *, const double *, double *, int, const double *, Shape, int32_t,
                                                const double *, double *);
template void launch_csr_spmv_t<float, float>(cudaStream_t, int32_t, int32_t, const int32_t *, const int32_t *,
                                              const float *, const float *, float *, int, const float *, Shape, int32_t,
                                              const float *, float *);
template void launch_csr_spmv_t<bf16, float>(cudaStream_t, int32_t, int32_t, const int32_t *, const int32_t *,
                                             const bf16 *, const float *, float *, int, const float *, Shape, int32_t,
                                             const float *, float *);

void launch_csr_spmv(cudaStream_t s, const Csr &A, const double *x, double *y, double alpha, const double *c0,
                     const double *ts, double *to) {
    int mode = c0 ? 1 : (alpha == 2.0 ? 2 : 0);
    launch_csr_spmv_t<double, double>(s, A.n, A.nnz, A.rp, A.ci, A.v, x, y, mode, c0, Shape(), A.n, ts, to);   // square
}

// FP64 -> FP32 (round to nearest) or FP64 -> FP32 -> BF16 (round to nearest even): the storage
// rounding of the mixed-precision form
__global__ void k_to_lower(const double *src, int64_t n, int st, void *dst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride) {
        float f = __double2float_rn(src[i]);
        if (st == ST_BF16) static_cast<bf16 *>(dst)[i] = __float2bfloat16_rn(f);
        else static_cast<float *>(dst)[i] = f;
    }
}
__global__ void k_d2f_vec(const double *a, float *b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}
__global__ void k_f2d_vec(const float *a, double *b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}
void launch_d2f(const Ctx *c, const double *a, float *b, int64_t n) {
    (k_d2f_vec<<<nblk(n, 256), 256, 0, c->stream>>>(a, b, n), note_launch());
}
void launch_f2d(const Ctx *c, const float *a, double *b, int64_t n) {
    (k_f2d_vec<<<nblk(n, 256), 256, 0, c->stream>>>(a, b, n), note_launch());
}

cptr_status to_lower(Ctx *c, const double *src, int64_t n, int st, void **dst) {
    size_t bytes = (size_t)(n > 0 ? n : 1) * (st == ST_BF16 ? 2 : 4);
    CPTR_TRY(dalloc(c, dst, bytes));
    if (n > 0) (k_to_lower<<<4 * 152, 256, 0, c->stream>>>(src, n, st, *dst), note_launch());
    return CPTR_OK;
}

// ------------------------------------------------------------------------------------------------
// restriction to / prolongation from the p-T unknowns (Sec. 3.2)
template <typename XT>
__global__ void k_gather_pt(int32_t n, int b, int ps, int ts, const double *v, XT *bp, XT *bT, const double *D,
                            const XT *sp, XT *tp, const XT *sT, XT *tT) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        double p = v[(int64_t)i * b + ps], t = v[(int64_t)i * b + ts];
        if (D)   // the decoupled right-hand side R G v
            for (int s = 0; s < b; ++s) {
                const double dp = D[((int64_t)i * 2) * b + s], dT = D[((int64_t)i * 2 + 1) * b + s];
                if (dp != 0.0) p = __dsub_rn(p, __dmul_rn(dp, v[(int64_t)i * b + s]));
                if (dT != 0.0) t = __dsub_rn(t, __dmul_rn(dT, v[(int64_t)i * b + s]));
            }
        bp[i] = (XT)p;
        bT[i] = (XT)t;
        // the first smoothing step of a V-cycle on bp or bT: t = D^{-1} b of its finest level
        if (tp) tp[i] = sp[i] * (XT)p;
        if (tT) tT[i] = sT[i] * (XT)t;
    }
}
template <typename XT>
void launch_gather_pt(const Ctx *c, const double *v, XT *bp, XT *bT, const XT *sp, XT *tp, const XT *sT, XT *tT) {
    (k_gather_pt<XT><<<nblk(c->n, 256), 256, 0, c->stream>>>(c->n, c->b, c->ps, c->ts, v, bp, bT, c->Ddec, sp, tp, sT,
                                                            tT),
     note_launch());
}
template void launch_gather_pt<double>(const Ctx *, const double *, double *, double *, const double *, double *,
                                       const double *, double *);
template void launch_gather_pt<float>(const Ctx *, const double *, float *, float *, const float *, float *,
                                      const float *, float *);

template <typename XT>
__global__ void k_scatter_pt(int32_t n, int b, int ps, int ts, const XT *dp, const XT *dT, double *x1) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        for (int q = 0; q < b; ++q) x1[(int64_t)i * b + q] = q == ps ? (double)dp[i] : (q == ts && dT ? (double)dT[i] : 0.0);
}
template <typename XT>
void launch_scatter_pt(const Ctx *c, const XT *dp, const XT *dT, double *x1) {
    (k_scatter_pt<XT><<<nblk(c->n, 256), 256, 0, c->stream>>>(c->n, c->b, c->ps, c->ts, dp, dT, x1), note_launch());
}
template void launch_scatter_pt<double>(const Ctx *, const double *, const double *, double *);
template void launch_scatter_pt<float>(const Ctx *, const float *, const float *, double *);

// mixed-precision stage-1 residual b1 = v - A' R_0^T [dp; dT] with FP32 values of A' (SELL-32)
template <int B>
__global__ void __launch_bounds__(512) k_sell_resid_pt32(int32_t n, const int64_t *__restrict__ off,
                                                          const int32_t *__restrict__ col,
                                                          const float *__restrict__ val, const double *__restrict__ v,
                                                          float *__restrict__ b1, int ps, int ts,
                                                          const float *__restrict__ dp, const float *__restrict__ dT) {
    int32_t row = blockIdx.x * blockDim.x + threadIdx.x;
    int32_t ch = row >> 5, lane = row & 31;
    if (row >= ((n + 31) & ~31)) return;
    const int64_t o0 = __ldg(off + ch), o1 = __ldg(off + ch + 1);
    float acc[B];
#pragma unroll
    for (int r = 0; r < B; ++r) acc[r] = 0.f;
    for (int64_t sl = o0; sl < o1; ++sl) {
        const int32_t cidx = __ldg(col + sl * 32 + lane);
        const float *a = val + sl * B * B * 32 + lane;
        const float xp = __ldg(dp + cidx);
        const float xt = dT ? __ldg(dT + cidx) : 0.f;
#pragma unroll
        for (int r = 0; r < B; ++r) {
            acc[r] = fmaf(__ldg(a + (r * B + ps) * 32), xp, acc[r]);
            if (dT) acc[r] = fmaf(__ldg(a + (r * B + ts) * 32), xt, acc[r]);
        }
    }
    if (row < n) {
#pragma unroll
        for (int r = 0; r < B; ++r) {
            int64_t oo = (int64_t)row * B + r;
            b1[oo] = (float)v[oo] - acc[r];
        }
    }
}
void launch_resid_pt32(const Ctx *c, const float *dp, const float *dT, const double *v, float *b1) {
    const int T = c->sell_shape.T;
    unsigned grid = nblk((int64_t)c->sell_nch * 32, T);
    if (c->b == 3)
        (k_sell_resid_pt32<3><<<grid, T, 0, c->stream>>>(c->n, c->sell_off, c->sell_col, c->sell_val32, v, b1, c->ps,
                                                          c->ts, dp, dT), note_launch());
    else
        (k_sell_resid_pt32<4><<<grid, T, 0, c->stream>>>(c->n, c->sell_off, c->sell_col, c->sell_val32, v, b1, c->ps,
                                                          c->ts, dp, dT), note_launch());
}

__global__ void k_sub(int32_t n, const double *a, const double *b, double *out) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] - b[i];
}
void launch_sub(cudaStream_t s, int32_t n, const double *a, const double *b, double *out) {
    (k_sub<<<nblk(n, 256), 256, 0, s>>>(n, a, b, out), note_launch());
}

// ------------------------------------------------------------------------------------------------
// Autotuner of the SELL kernels: threads per block in {64, 128, 256, 512}, each timed with CUDA
// events over 5 launches of y = A' x after one warm-up launch; the fastest is kept (cached by the
// matrix size, so repeated set-ups of one workload tune once).
cptr_status sell_autotune(Ctx *c) {
    const uint64_t key = (uint64_t)7 << 60 | (uint64_t)c->b << 56 | (uint64_t)(c->sell_nvals & ((1ull << 56) - 1));
    auto it = c->tune_cache.find(key);
    if (it != c->tune_cache.end()) {
        c->sell_shape = it->second;
        return CPTR_OK;
    }
    cudaEvent_t e0, e1;
    CPTR_CUDA_TRY(c, cudaEventCreate(&e0));
    CPTR_CUDA_TRY(c, cudaEventCreate(&e1));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(c->zcur, 0, sizeof(double) * (size_t)c->n * c->b, c->stream));
    Shape best;
    float best_ms = 1e30f;
    for (int T : {64, 128, 256, 512}) {
        c->sell_shape.T = (int16_t)T;
        launch_bsr_spmv(c, c->zcur, c->w);
        cudaEventRecord(e0, c->stream);
        for (int r = 0; r < 5; ++r) launch_bsr_spmv(c, c->zcur, c->w);
        cudaEventRecord(e1, c->stream);
        CPTR_CUDA_TRY(c, cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) { best_ms = ms; best = c->sell_shape; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->sell_shape = best;
    c->tune_cache[key] = best;
    CPTR_CUDA_TRY(c, cudaGetLastError());
    return CPTR_OK;
}

}  // namespace cptr
