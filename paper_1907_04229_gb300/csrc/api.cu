// C ABI of the CPTR library (declared in include/cptr.h): argument validation, set-up
// orchestration (decoupling, p-T extraction, two AMG hierarchies, ILU(0)), and the solve.
#include <cuda_runtime.h>
#include <string.h>

#include <stddef.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <thread>

#include "common.cuh"

using namespace cptr;

namespace {

bool host_or_device_copy(Ctx *c, void *dst, const void *src, size_t bytes, int on_device, cudaMemcpyKind to) {
    cudaError_t e;
    if (on_device) e = cudaMemcpyAsync(dst, src, bytes, to == cudaMemcpyDeviceToHost ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream);
    else e = cudaMemcpyAsync(dst, src, bytes, to == cudaMemcpyDeviceToHost ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice, c->stream);
    return e == cudaSuccess;
}

void release_setup(Ctx *c) {
    dfree(c->rp); dfree(c->ci); dfree(c->diag); dfree(c->A); dfree(c->W);
    dfree(c->sell_off); dfree(c->sell_col); dfree(c->sell_val);
    c->sell_off = nullptr; c->sell_col = nullptr; c->sell_val = nullptr;
    dfree(c->App); dfree(c->ApT); dfree(c->ATp); dfree(c->St); dfree(c->Ddec);
    c->Ddec = nullptr;
    dfree(c->lf_base); dfree(c->lf_sat); dfree(c->lf_s);
    c->rp = c->ci = c->diag = nullptr;
    c->A = c->W = c->App = c->ApT = c->ATp = c->St = nullptr;
    c->lf_base = c->lf_sat = c->lf_s = nullptr;
    c->schur_used = 0;
    amg_free(c->hp);
    amg_free(c->hT);
    ilu_free(c);
    double **vecs[] = {&c->bp, &c->bT, &c->xp, &c->dp, &c->dT, &c->t1, &c->b1, &c->V, &c->Z, &c->w, &c->bw, &c->xw,
                       &c->vcur, &c->zcur, &c->b00, &c->x00};
    for (double **p : vecs) { dfree(*p); *p = nullptr; }
    float **vecs32[] = {&c->ApT32, &c->ATp32, &c->sell_val32, &c->bp32, &c->bT32, &c->xp32, &c->dp32, &c->dT32,
                        &c->t132, &c->b132, &c->b0032, &c->x0032};
    for (float **p : vecs32) { dfree(*p); *p = nullptr; }
    if (c->graph_exec) {
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
    }
    if (c->cycle_exec) {
        cudaGraphExecDestroy(c->cycle_exec);
        c->cycle_exec = nullptr;
    }
    free_batch(c);
    c->sell_shape = Shape();
    c->tl_best_ty = c->tl_best_tz = 0;
    c->sf_grid = 4 * 152;
    c->sf_sleep = 20;
    c->ready = false;
}

// The pattern is checked on the device: per row, column indices in [0, n), strictly ascending,
// and a diagonal block.  The first failing row (and its first failing entry) is kept as
// row * 4 + kind (0 out of range, 1 not ascending, 2 no diagonal) by an atomic minimum.
__global__ void k_validate_rows(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                int32_t *diag, unsigned long long *err) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t d = -1;
    int kind = -1;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
        const int32_t j = ci[k];
        if (j < 0 || j >= n) { kind = 0; break; }
        if (k > rp[i] && ci[k - 1] >= j) { kind = 1; break; }
        if (j == i) d = k;
    }
    if (kind < 0 && d < 0) kind = 2;
    diag[i] = d;
    if (kind >= 0) atomicMin(err, ((unsigned long long)i << 2) | (unsigned long long)kind);
}

// row_ptr on the host (already checked to start at 0 and end at nnzb), col_idx on the device
cptr_status validate_pattern(Ctx *c, int32_t n) {
    const std::vector<int32_t> &rp = c->h_rp;
    for (int32_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) return c->fail(CPTR_EINVAL, "row_ptr decreases at row " + std::to_string(i));
    unsigned long long *err = nullptr, h_err = ~0ULL;
    CPTR_TRY(dalloc_t(c, &err, 1));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(err, 0xFF, sizeof(unsigned long long), c->stream));
    (k_validate_rows<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, c->rp, c->ci, c->diag, err), note_launch());
    const cptr_status cs = copy_to_host(c, &h_err, err, sizeof(h_err));
    dfree(err);
    CPTR_TRY(cs);
    if (h_err == ~0ULL) return CPTR_OK;
    const std::string row = std::to_string((long long)(h_err >> 2));
    switch ((int)(h_err & 3)) {
        case 0: return c->fail(CPTR_EINVAL, "col_idx out of range in row " + row);
        case 1: return c->fail(CPTR_EINVAL, "col_idx not strictly ascending in row " + row);
        default: return c->fail(CPTR_EINVAL, "missing diagonal block in row " + row);
    }
}

}  // namespace

// column indices and pivot positions on the host, copied from the device once per set-up (the
// multicolour ordering and the chunked sweep tables are built on the host)
cptr_status cptr::host_pattern(Ctx *c) {
    if (c->h_ci.size() == (size_t)c->nnzb && c->h_diag.size() == (size_t)c->n) return CPTR_OK;
    c->h_ci.assign((size_t)c->nnzb, 0);
    c->h_diag.assign((size_t)c->n, 0);
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->h_diag.data(), c->diag, sizeof(int32_t) * c->n, cudaMemcpyDeviceToHost, c->stream));
    return copy_to_host(c, c->h_ci.data(), c->ci, sizeof(int32_t) * c->nnzb);
}

namespace {

cptr_status clear_wait_flag(Ctx *c);
cptr_status check_wait_flag(Ctx *c);

cptr_status do_setup(Ctx *c, int32_t n, int32_t b, const int32_t *row_ptr, const int32_t *col_idx, const double *vals,
                     const int32_t *kind, const double *W, const double *st, int on_device, int kind_on_device) {
    if (n <= 0) return c->fail(CPTR_EINVAL, "n_cells must be positive");
    if (b != 3 && b != 4) return c->fail(CPTR_EINVAL, "b must be 3 or 4");
    if (!row_ptr || !col_idx || !vals || !kind) return c->fail(CPTR_EINVAL, "row_ptr, col_idx, vals, unknown_kind are required");
    int32_t hk[4];
    if (kind_on_device) CPTR_TRY(copy_to_host(c, hk, kind, sizeof(int32_t) * b));
    else memcpy(hk, kind, sizeof(int32_t) * b);
    int ps = -1, ts = -1;
    for (int q = 0; q < b; ++q) {
        if (hk[q] == CPTR_U_P) { if (ps >= 0) return c->fail(CPTR_EINVAL, "more than one pressure slot"); ps = q; }
        else if (hk[q] == CPTR_U_T) { if (ts >= 0) return c->fail(CPTR_EINVAL, "more than one temperature slot"); ts = q; }
        else if (hk[q] != CPTR_U_SAT) return c->fail(CPTR_EINVAL, "unknown_kind entries must be P, T or SAT");
    }
    if (ps < 0 || ts < 0) return c->fail(CPTR_EINVAL, "unknown_kind needs one P and one T slot");
    release_setup(c);
    for (double &v : c->prof.setup_ms) v = 0.0;
    auto t0 = std::chrono::steady_clock::now();
    // pattern to the host for validation and level scheduling
    c->h_rp.assign((size_t)n + 1, 0);
    if (on_device) CPTR_TRY(copy_to_host(c, c->h_rp.data(), row_ptr, sizeof(int32_t) * ((size_t)n + 1)));
    else memcpy(c->h_rp.data(), row_ptr, sizeof(int32_t) * ((size_t)n + 1));
    int32_t nnzb = c->h_rp[n];
    if (nnzb <= 0 || c->h_rp[0] != 0) return c->fail(CPTR_EINVAL, "row_ptr must start at 0 and end at nnzb > 0");
    c->h_ci.clear();
    c->h_diag.clear();
    c->n = n; c->b = b; c->ps = ps; c->ts = ts; c->nnzb = nnzb;
    const size_t bb = (size_t)b * b;
    CPTR_TRY(dalloc_t(c, &c->rp, (size_t)n + 1));
    CPTR_TRY(dalloc_t(c, &c->ci, (size_t)nnzb));
    CPTR_TRY(dalloc_t(c, &c->diag, (size_t)n));
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->rp, c->h_rp.data(), sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, c->stream));
    if (!host_or_device_copy(c, c->ci, col_idx, sizeof(int32_t) * nnzb, on_device, cudaMemcpyHostToDevice))
        return c->fail(CPTR_ECUDA, "copy of col_idx failed");
    CPTR_TRY(validate_pattern(c, n));
    double *Araw = nullptr;
    CPTR_TRY(dalloc_t(c, &Araw, nnzb * bb));
    CPTR_TRY(dalloc_t(c, &c->A, nnzb * bb));
    if (!host_or_device_copy(c, Araw, vals, sizeof(double) * nnzb * bb, on_device, cudaMemcpyHostToDevice))
        return c->fail(CPTR_ECUDA, "copy of vals failed");
    if (W) {
        CPTR_TRY(dalloc_t(c, &c->W, (size_t)n * bb));
        if (!host_or_device_copy(c, c->W, W, sizeof(double) * n * bb, on_device, cudaMemcpyHostToDevice))
            return c->fail(CPTR_ECUDA, "copy of row_weights failed");
    }
    // the caller's S~_T is used by CPTR_SCHUR_GIVEN, and is the fallback of CPTR_SCHUR_LEARNED
    const bool use_st = st && c->o.schur != CPTR_SCHUR_ATT;
    CPTR_TRY(dalloc_t(c, &c->St, (size_t)nnzb));
    if (use_st) {
        if (!host_or_device_copy(c, c->St, st, sizeof(double) * nnzb, on_device, cudaMemcpyHostToDevice))
            return c->fail(CPTR_ECUDA, "copy of st_vals failed");
    }
    // finite values
    CPTR_CUDA_TRY(c, cudaMemsetAsync(c->flag, 0, sizeof(int32_t), c->stream));
    launch_check_finite(c, Araw, (int64_t)nnzb * bb, c->flag);
    if (c->W) launch_check_finite(c, c->W, (int64_t)n * bb, c->flag);
    if (use_st) launch_check_finite(c, c->St, nnzb, c->flag);
    int32_t bad = 0;
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(&bad, c->flag, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (bad) { dfree(Araw); return c->fail(CPTR_EINVAL, "non-finite value in vals, row_weights or st_vals"); }
    // A' = W A, then the scalar p-T blocks on the cell pattern (those of G A' for a decoupled stage 1)
    launch_decouple(c, Araw, c->W, c->A);
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    dfree(Araw);
    if (c->o.decouple != CPTR_DECOUPLE_NONE) CPTR_TRY(decoupling_setup(c));
    CPTR_TRY(dalloc_t(c, &c->App, (size_t)nnzb));
    CPTR_TRY(dalloc_t(c, &c->ApT, (size_t)nnzb));
    CPTR_TRY(dalloc_t(c, &c->ATp, (size_t)nnzb));
    launch_extract(c, ps, ps, c->App);
    launch_extract(c, ps, ts, c->ApT);
    launch_extract(c, ts, ps, c->ATp);
    if (!use_st) launch_extract(c, ts, ts, c->St);
    c->schur_used = use_st ? CPTR_SCHUR_GIVEN : CPTR_SCHUR_ATT;
    CPTR_TRY(learned_prepare(c));
    CPTR_CUDA_TRY(c, cudaGetLastError());
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->prof.setup_ms[SETUP_INPUTS] +=
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (c->o.schur == CPTR_SCHUR_LEARNED) {
        // S~_T = diag(s) S~_T from the network; on rejection the S~_T above stays
        double tl = host_ms();
        bool used = false;
        CPTR_TRY(learned_schur(c, &used));
        if (used) c->schur_used = CPTR_SCHUR_LEARNED;
        setup_tick(c, SETUP_OTHER, &tl);
    }
    int s1 = c->o.stage1;
    // S~_diag = A_TT - A_Tp diag(A_pp)^{-1} A_pT (Sec. 3.3.1), on its own (wider) pattern
    Csr Sd;
    if (c->o.schur == CPTR_SCHUR_DIAG && s1 != CPTR_STAGE1_NONE && s1 != CPTR_STAGE1_CPR && s1 != CPTR_STAGE1_UAMG) {
        CPTR_TRY(schur_diag(c, Sd));
        c->schur_used = CPTR_SCHUR_DIAG;
    }
    // The hierarchies are independent of one another: each is built by a host thread of its own
    // (a context view with its own stream, fork event, scratch flag and scan buffer).  The ILU(0)
    // factors follow on this thread once both are built: building them at the same time gave no
    // gain on 200k cells (every part of the set-up slowed down in proportion), and on 2M cells the
    // ILU set-up and the coarsening then stalled each other for ~0.4 s in most set-ups.
    struct HierJob {
        Hier *h;
        const int32_t *rp, *ci;
        const double *v;
        int32_t n;
        const int32_t *fn;
        int32_t np;
    };
    std::vector<HierJob> jobs;
    Csr A00;
    int32_t *fn00 = nullptr;
    if (s1 == CPTR_STAGE1_UAMG) {
        // unknown-based AMG (Sec. 3.4) on A_00 in unknown-wise order, kept in the pressure slot
        CPTR_TRY(build_a00(c, A00, &fn00));
        jobs.push_back({&c->hp, A00.rp, A00.ci, A00.v, 2 * n, fn00, n});
    } else if (s1 != CPTR_STAGE1_NONE) {
        jobs.push_back({&c->hp, c->rp, c->ci, c->App, n, nullptr, 0});
        if (s1 != CPTR_STAGE1_CPR)
            jobs.push_back(Sd.v ? HierJob{&c->hT, Sd.rp, Sd.ci, Sd.v, n, nullptr, 0}
                                : HierJob{&c->hT, c->rp, c->ci, c->St, n, nullptr, 0});
    }
    if (!c->coarse_stream && !jobs.empty())
        CPTR_CUDA_TRY(c, cudaStreamCreateWithFlags(&c->coarse_stream, cudaStreamNonBlocking));
    const size_t nj = jobs.size();
    std::vector<Ctx> wc(nj);
    std::vector<cptr_status> st_w(nj, CPTR_OK);
    for (size_t q = 0; q < nj; ++q) {
        if (!c->amg_stream[q]) CPTR_CUDA_TRY(c, cudaStreamCreateWithFlags(&c->amg_stream[q], cudaStreamNonBlocking));
        if (!c->amg_fork[q]) CPTR_CUDA_TRY(c, cudaEventCreateWithFlags(&c->amg_fork[q], cudaEventDisableTiming));
        Ctx &w = wc[q];
        w.o = c->o;
        w.stream = c->amg_stream[q];
        w.pool = c->pool;
        w.coarse_stream = c->coarse_stream;
        w.side_fork = c->amg_fork[q];
        CPTR_TRY(dalloc_t(c, &w.flag, 4));
    }
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));   // inputs and allocations are ready
    // a host exception on any thread becomes a status: the workers catch their own, and this
    // thread joins the workers before any exception of its own leaves this scope
    std::vector<std::thread> workers;
    for (size_t q = 0; q < nj; ++q)
        workers.emplace_back([&, q] {
            Ctx &w = wc[q];
            const HierJob &j = jobs[q];
            CtxScope ws(&w);
            try {
                st_w[q] = amg_setup(&w, *j.h, j.rp, j.ci, j.v, j.n, j.fn, j.np);
            } catch (const std::bad_alloc &) {
                st_w[q] = w.fail(CPTR_ENOMEM, "host allocation failed");
            } catch (...) {
                st_w[q] = w.fail(CPTR_EINVAL, "unexpected host exception");
            }
            dfree(w.scan_tmp);
            w.scan_tmp = nullptr;
            cudaStreamSynchronize(w.stream);
        });
    auto join_all = [&] {
        for (auto &t : workers) t.join();
        workers.clear();
        for (Ctx &w : wc) {
            dfree(w.flag);
            w.flag = nullptr;
        }
        csr_free(A00);
        dfree(fn00);
        fn00 = nullptr;
        csr_free(Sd);
    };
    join_all();
    for (const Ctx &w : wc)
        for (int q = 0; q < kSetupPhases; ++q) c->prof.setup_ms[q] += w.prof.setup_ms[q];
    for (size_t q = 0; q < nj; ++q)
        if (st_w[q] != CPTR_OK) return c->fail(st_w[q], wc[q].err);
    if (c->o.stage2 == CPTR_STAGE2_ILU0) CPTR_TRY(ilu_setup(c));
    // the coarsest inverses ran on the coarse stream meanwhile
    CPTR_TRY(amg_coarsest_wait(c, c->hp));
    CPTR_TRY(amg_coarsest_wait(c, c->hT));
    double t2 = host_ms();
    // A' for the solve in the SELL-32 layout; the BSR copy is not needed after set-up
    CPTR_TRY(sell_build(c));
    if (c->o.precision == CPTR_PREC_MIXED) {
        // FP32/BF16 copies of the preconditioner's operators (the FP64 set-up is rounded once)
        if (s1 != CPTR_STAGE1_NONE) CPTR_TRY(amg_lower_precision(c, c->hp));
        if (uses_T(s1)) CPTR_TRY(amg_lower_precision(c, c->hT));
        CPTR_TRY(to_lower(c, c->ApT, nnzb, ST_F32, (void **)&c->ApT32));
        CPTR_TRY(to_lower(c, c->ATp, nnzb, ST_F32, (void **)&c->ATp32));
        CPTR_TRY(to_lower(c, c->sell_val, c->sell_nvals, ST_F32, (void **)&c->sell_val32));
        for (float **p : {&c->bp32, &c->bT32, &c->xp32, &c->dp32, &c->dT32, &c->t132}) CPTR_TRY(dalloc_t(c, p, (size_t)n));
        CPTR_TRY(dalloc_t(c, &c->b132, (size_t)n * b));
    }
    if (s1 != CPTR_STAGE1_NONE) CPTR_TRY(amg_fuse_setup(c, c->hp));
    if (uses_T(s1)) CPTR_TRY(amg_fuse_setup(c, c->hT));
    dfree(c->A);
    c->A = nullptr;
    setup_tick(c, SETUP_LAYOUT, &t2);
    // work vectors
    const size_t nb = (size_t)n * b;
    const int m = c->o.restart;
    for (double **p : {&c->bp, &c->bT, &c->xp, &c->dp, &c->dT, &c->t1}) CPTR_TRY(dalloc_t(c, p, (size_t)n));
    if (s1 == CPTR_STAGE1_UAMG) {   // [b_p; b_T] and [d_p; d_T] of the unknown-based V-cycle
        CPTR_TRY(dalloc_t(c, &c->b00, 2 * (size_t)n));
        CPTR_TRY(dalloc_t(c, &c->x00, 2 * (size_t)n));
        if (c->o.precision == CPTR_PREC_MIXED) {
            CPTR_TRY(dalloc_t(c, &c->b0032, 2 * (size_t)n));
            CPTR_TRY(dalloc_t(c, &c->x0032, 2 * (size_t)n));
        }
    }
    for (double **p : {&c->b1, &c->w, &c->bw, &c->xw, &c->vcur, &c->zcur}) CPTR_TRY(dalloc_t(c, p, nb));
    CPTR_TRY(dalloc_t(c, &c->V, nb * (m + 1)));
    CPTR_TRY(dalloc_t(c, &c->Z, nb * m));
    if (c->o.autotune) {
        double ta = host_ms();
        if (s1 != CPTR_STAGE1_NONE) CPTR_TRY(amg_autotune(c, c->hp));
        if (uses_T(s1)) CPTR_TRY(amg_autotune(c, c->hT));
        CPTR_TRY(sell_autotune(c));
        if (c->o.stage2 == CPTR_STAGE2_ILU0) {
            CPTR_TRY(clear_wait_flag(c));
            CPTR_TRY(ilu_autotune(c));
            CPTR_TRY(check_wait_flag(c));
        }
        setup_tick(c, SETUP_OTHER, &ta);
    } else if (c->o.csr_lanes) {
        for (Hier *h : {&c->hp, &c->hT})
            for (int l = 0; l < h->nlev; ++l) {
                Level &L = h->L[l];
                L.sh_A.G = L.sh_PT.G = L.sh_P.G = (int16_t)c->o.csr_lanes;
            }
    }
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    CPTR_CUDA_TRY(c, cudaGetLastError());
    c->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    c->ready = true;
    return CPTR_OK;
}

template <typename F>
cptr_status guarded(cptr_ctx *ctx, F &&f) {
    if (!ctx) return CPTR_EINVAL;
    CtxScope scope(&ctx->c);
    try {
        ctx->c.err.clear();
        const cptr_status st = f(&ctx->c);
        const cptr_status ck = check_report(&ctx->c);   // the bounds-checking build only
        return ck != CPTR_OK ? ck : st;
    } catch (const std::bad_alloc &) {
        return ctx->c.fail(CPTR_ENOMEM, "host allocation failed");
    } catch (...) {
        return ctx->c.fail(CPTR_EINVAL, "unexpected host exception");
    }
}

cptr_status need_ready(Ctx *c) {
    if (!c->ready) return c->fail(CPTR_ESTATE, "no successful cptr_setup on this context");
    return CPTR_OK;
}

cptr_status sync(Ctx *c) {
    CPTR_CUDA_TRY(c, cudaGetLastError());
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return CPTR_OK;
}

// component calls that run the ILU sweeps: clear the wait flag before, check it after
cptr_status clear_wait_flag(Ctx *c) {
    CPTR_CUDA_TRY(c, cudaMemsetAsync(reinterpret_cast<char *>(c->ks) + offsetof(KState, wait_err), 0, sizeof(int32_t),
                                     c->stream));
    return CPTR_OK;
}
cptr_status check_wait_flag(Ctx *c) {
    int32_t w = 0;
    CPTR_TRY(copy_to_host(c, &w, reinterpret_cast<char *>(c->ks) + offsetof(KState, wait_err), sizeof(int32_t)));
    if (w) return c->fail(CPTR_ETIMEOUT, "ILU(0) sweep: a bounded wait gave up");
    return CPTR_OK;
}

// a device view of a caller array: the array itself (on_device) or a device copy of a host array
template <typename T>
struct DevIn {
    const T *p = nullptr;
    T *own = nullptr;
    ~DevIn() { dfree(own); }
    cptr_status init(Ctx *c, const T *src, size_t count, int on_device) {
        if (on_device) { p = src; return CPTR_OK; }
        CPTR_TRY(dalloc_t(c, &own, count));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(own, src, sizeof(T) * count, cudaMemcpyHostToDevice, c->stream));
        p = own;
        return CPTR_OK;
    }
};
// a device output for a caller array, copied back to the host by finish()
template <typename T>
struct DevOut {
    T *p = nullptr, *own = nullptr, *host = nullptr;
    size_t count = 0;
    ~DevOut() { dfree(own); }
    cptr_status init(Ctx *c, T *dst, size_t n, int on_device) {
        count = n;
        if (on_device) { p = dst; return CPTR_OK; }
        CPTR_TRY(dalloc_t(c, &own, n));
        p = own;
        host = dst;
        return CPTR_OK;
    }
    cptr_status finish(Ctx *c) {
        if (host) return copy_to_host(c, host, own, sizeof(T) * count);
        return sync(c);
    }
};
}  // namespace

extern "C" {

cptr_status cptr_default_options(cptr_options *o) {
    if (!o) return CPTR_EINVAL;
    memset(o, 0, sizeof(*o));
    o->stage1 = CPTR_STAGE1_FULL;
    o->stage2 = CPTR_STAGE2_ILU0;
    o->schur = CPTR_SCHUR_GIVEN;
    o->smoother = CPTR_SMOOTH_L1;
    o->omega = 2.0 / 3.0;
    o->theta = 0.25;
    o->n_coarse = 256;
    o->max_levels = 25;
    o->restart = 30;
    o->max_it = 1000;
    o->dense_max = 1024;
    o->seed = 0;
    o->precision = CPTR_PREC_FP64;
    o->check_every = 1;
    o->use_graph = 1;
    o->stream = nullptr;
    return CPTR_OK;
}

cptr_status cptr_create(cptr_ctx **out, const cptr_options *opt) {
    if (!out) return CPTR_EINVAL;
    *out = nullptr;
    cptr_options o;
    if (opt) o = *opt;
    else cptr_default_options(&o);
    if (o.restart < 1 || o.restart > kMaxRestart || o.max_it < 0 || o.max_levels < 1 || o.dense_max < 1 || o.dense_max > 25600 ||
        o.stage1 < 0 || o.stage1 > CPTR_STAGE1_UAMG || o.stage2 < 0 || o.stage2 > CPTR_STAGE2_NONE ||
        o.smoother < 0 || o.smoother > CPTR_SMOOTH_JACOBI || o.schur < CPTR_SCHUR_GIVEN ||
        o.schur > CPTR_SCHUR_DIAG || o.precision < CPTR_PREC_FP64 ||
        o.precision > CPTR_PREC_MIXED ||
        o.ilu_order < CPTR_ILU_NATURAL || o.ilu_order > CPTR_ILU_MULTICOLOR || o.ilu_sweep < 0 || o.ilu_sweep > 4 || o.use_graph < 0 || o.use_graph > 2 ||
        o.tile_y < 0 || o.tile_z < 0 || (size_t)o.tile_y * o.tile_z > 64 || o.decouple < CPTR_DECOUPLE_NONE ||
        o.decouple > CPTR_DECOUPLE_TI ||
        (o.decouple != CPTR_DECOUPLE_NONE && o.stage1 != CPTR_STAGE1_CPR && o.stage1 != CPTR_STAGE1_UAMG) ||
        o.ilu_fill < 0 || o.ilu_fill > 1 || (o.ilu_fill == 1 && o.ilu_order == CPTR_ILU_MULTICOLOR) ||
        o.csr_lanes < 0 || o.csr_lanes > 32 || (o.csr_lanes & (o.csr_lanes - 1)) || o.ilu_group < 0 || o.ilu_group == 1 ||
        o.ilu_group > 4 || (o.ilu_lanes != 0 && o.ilu_lanes != 4 && o.ilu_lanes != 8 && o.ilu_lanes != 16))
        return CPTR_EINVAL;
    cptr_ctx *ctx = new (std::nothrow) cptr_ctx();
    if (!ctx) return CPTR_ENOMEM;
    Ctx *c = &ctx->c;
    c->o = o;
    c->stream = (cudaStream_t)o.stream;
    CtxScope scope(c);
    {
        // a stream-ordered pool for this context; freed blocks stay reserved for the next set-up
        int dev = 0;
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        if (cudaGetDevice(&dev) == cudaSuccess) {
            props.location.id = dev;
            if (cudaMemPoolCreate(&c->pool, &props) == cudaSuccess) {
                uint64_t keep = UINT64_MAX;
                cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
                // the set-up allocates from several streams (two host threads, the factorisation
                // and the coarsest inverses on streams of their own): memory freed on one stream is
                // reused on another only once the free has completed, never by making the
                // allocating stream wait on the other one's pending work
                int no = 0;
                cudaMemPoolSetAttribute(c->pool, cudaMemPoolReuseAllowInternalDependencies, &no);
            } else {
                c->pool = nullptr;   // fall back to cudaMalloc
            }
        }
    }
    cptr_status s = CPTR_OK;
    if ((s = dalloc_t(c, &c->ks, 1)) != CPTR_OK || (s = dalloc_t(c, &c->flag, 4)) != CPTR_OK ||
        (s = dalloc_t(c, &c->never, 1)) != CPTR_OK ||
        (s = dalloc_t(c, &c->partial, (size_t)kRedBlocks * (kMaxRestart + 2))) != CPTR_OK) {
        cptr_destroy(ctx);
        return s;
    }
    if (cudaMallocHost((void **)&c->ks_host, sizeof(KState)) != cudaSuccess) {
        c->ks_host = nullptr;
        cptr_destroy(ctx);
        return CPTR_ENOMEM;
    }
    amg_preload();
    *out = ctx;
    return CPTR_OK;
}

void cptr_destroy(cptr_ctx *ctx) {
    if (!ctx) return;
    Ctx *c = &ctx->c;
    {
        CtxScope scope(c);
        cudaStreamSynchronize(c->stream);
        if (c->side_stream) cudaStreamSynchronize(c->side_stream);
        if (c->coarse_stream) cudaStreamSynchronize(c->coarse_stream);
        for (cudaStream_t as : c->amg_stream)
            if (as) cudaStreamSynchronize(as);
        release_setup(c);
        ilu_sym_free(c);
        dfree(c->part);
        c->part = nullptr;
        dfree(c->ks); dfree(c->flag); dfree(c->partial); dfree(c->scan_tmp); dfree(c->never); dfree(c->ilu_flags);
        dfree(c->mlp);
        model_free(c);
        cudaStreamSynchronize(c->stream);
    }
    if (c->pool) cudaMemPoolDestroy(c->pool);
    if (c->ks_host) cudaFreeHost(c->ks_host);
    for (cudaEvent_t e : c->prof.ev) cudaEventDestroy(e);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->side_stream) cudaStreamDestroy(c->side_stream);
    if (c->coarse_stream) cudaStreamDestroy(c->coarse_stream);
    for (cudaStream_t as : c->amg_stream)
        if (as) cudaStreamDestroy(as);
    for (cudaEvent_t ae : c->amg_fork)
        if (ae) cudaEventDestroy(ae);
    if (c->side_fork) cudaEventDestroy(c->side_fork);
    if (c->side_join) cudaEventDestroy(c->side_join);
    for (Hier *h : {&c->hp, &c->hT})
        if (h->gj_done) cudaEventDestroy(h->gj_done);
    delete ctx;
}

const char *cptr_last_error(const cptr_ctx *ctx) { return ctx ? ctx->c.err.c_str() : "null context"; }

cptr_status cptr_setup(cptr_ctx *ctx, int32_t n_cells, int32_t b, const int32_t *row_ptr, const int32_t *col_idx,
                       const double *vals, const int32_t *unknown_kind, const double *row_weights,
                       const double *st_vals, int32_t on_device) {
    return guarded(ctx, [&](Ctx *c) {
        cptr_status s = do_setup(c, n_cells, b, row_ptr, col_idx, vals, unknown_kind, row_weights, st_vals, on_device,
                                 on_device);
        if (s != CPTR_OK) {
            std::string keep = c->err;
            cudaStreamSynchronize(c->stream);
            release_setup(c);
            c->err = keep;
        }
        return s;
    });
}

cptr_status cptr_solve(cptr_ctx *ctx, const double *rhs, double *x, double rtol, cptr_stats *st, int32_t on_device) {
    return guarded(ctx, [&](Ctx *c) {
        CPTR_TRY(need_ready(c));
        if (!rhs || !x) return c->fail(CPTR_EINVAL, "rhs and x are required");
        if (!(rtol >= 0.0)) return c->fail(CPTR_EINVAL, "rtol must be >= 0");
        const size_t nb = (size_t)c->n * c->b;
        cudaEvent_t e0, e1;
        CPTR_CUDA_TRY(c, cudaEventCreate(&e0));
        CPTR_CUDA_TRY(c, cudaEventCreate(&e1));
        CPTR_CUDA_TRY(c, cudaEventRecord(e0, c->stream));
        const double *rhs_dev = rhs;
        if (!on_device) {
            CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->xw, rhs, sizeof(double) * nb, cudaMemcpyHostToDevice, c->stream));
            rhs_dev = c->xw;
        }
        launch_weight_vec(c, c->W, rhs_dev, c->bw);
        double *xd = on_device ? x : c->xw;
        prof_reset(c);
        cptr_status s = fgmres_solve(c, c->bw, xd, rtol, st);
        if (!on_device && (s == CPTR_OK || s == CPTR_NOT_CONVERGED))
            CPTR_CUDA_TRY(c, cudaMemcpyAsync(x, c->xw, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->stream));
        CPTR_CUDA_TRY(c, cudaEventRecord(e1, c->stream));
        CPTR_CUDA_TRY(c, cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        CPTR_TRY(prof_collect(c));
        if (st) {
            st->solve_ms = ms;
            st->setup_ms = c->setup_ms;
            st->levels_p = c->hp.nlev;
            st->levels_T = c->hT.nlev;
            st->op_complexity_p = c->hp.op_complexity;
            st->op_complexity_T = c->hT.op_complexity;
            st->schur_used = c->schur_used;
        }
        return s;
    });
}

cptr_status cptr_apply_matrix(cptr_ctx *ctx, const double *x, double *y) {
    return guarded(ctx, [&](Ctx *c) {
        CPTR_TRY(need_ready(c));
        launch_bsr_spmv(c, x, y);
        return sync(c);
    });
}

cptr_status cptr_apply_weights(cptr_ctx *ctx, const double *rhs, double *out) {
    return guarded(ctx, [&](Ctx *c) {
        CPTR_TRY(need_ready(c));
        launch_weight_vec(c, c->W, rhs, out);
        return sync(c);
    });
}

cptr_status cptr_apply_stage1(cptr_ctx *ctx, const double *v, double *x1) {
    return guarded(ctx, [&](Ctx *c) {
        CPTR_TRY(need_ready(c));
        if (c->o.precision == CPTR_PREC_MIXED) {
            const float *dp, *dT;
            apply_stage1_32(c, v, &dp, &dT);
            if (dp) launch_scatter_pt<float>(c, dp, dT, x1);
            else CPTR_CUDA_TRY(c, cudaMemsetAsync(x1, 0, sizeof(double) * c->n * c->b, c->stream));
        } else {
            const double *dp, *dT;
            apply_stage1(c, v, &dp, &dT);
            if (dp) launch_scatter_pt<double>(c, dp, dT, x1);
            else CPTR_CUDA_TRY(c, cudaMemsetAsync(x1, 0, sizeof(double) * c->n * c->b, c->stream));
        }
        return sync(c);
    });
}

cptr_status cptr_apply_ilu(cptr_ctx *ctx, const double *r, double *z) {
    return guarded(ctx, [&](Ctx *c) {
        CPTR_TRY(need_ready(c));
        if (c->o.stage2 != CPTR_STAGE2_ILU0) return c->fail(CPTR_ESTATE, "ILU(0) was not set up");
        CPTR_TRY(clear_wait_flag(c));
        ilu_apply(c, r, z, nullptr, nullptr);
        CPTR_TRY(sync(c));
        return check_wait_flag(c);
    });
}

cptr_status cptr_apply_precond(cptr_ctx *ctx, const double *v, double *z) {
    return guarded(ctx, [&](Ctx *c) {
        CPTR_TRY(need_ready(c));
        CPTR_TRY(clear_wait_flag(c));
        apply_precond(c, v, z);
        CPTR_TRY(sync(c));
        return check_wait_flag(c);
    });
}

cptr_status cptr_apply_vcycle(cptr_ctx *ctx, int32_t which, const double *b, double *x) {
    return guarded(ctx, [&](Ctx *c) {
        CPTR_TRY(need_ready(c));
        if (which < 0 || which > 1) return c->fail(CPTR_EINVAL, "no such AMG hierarchy");
        const Hier &h = which == 0 ? c->hp : c->hT;
        if (h.nlev == 0) return c->fail(CPTR_EINVAL, "no such AMG hierarchy");
        if (c->o.precision == CPTR_PREC_MIXED) {   // FP64 in and out, FP32 cycle
            const int32_t len = h.L[0].A.n;      // n, or 2n for the unknown-based A_00 hierarchy
            float *b32 = len > c->n ? c->b0032 : c->bp32, *x32 = len > c->n ? c->x0032 : c->dp32;
            launch_d2f(c, b, b32, len);
            amg_vcycle32(c, h, b32, x32);
            launch_f2d(c, x32, x, len);
        } else {
            amg_vcycle(c, h, b, x);
        }
        return sync(c);
    });
}

cptr_status cptr_hierarchy_info(cptr_ctx *ctx, int32_t which, int32_t *nlev, int32_t *info) {
    return guarded(ctx, [&](Ctx *c) {
        CPTR_TRY(need_ready(c));
        if (!nlev || !info || which < 0 || which > 1) return c->fail(CPTR_EINVAL, "bad arguments");
        const Hier &h = which == 0 ? c->hp : c->hT;
        *nlev = h.nlev;
        for (int l = 0; l < h.nlev; ++l) {
            info[4 * l + 0] = h.L[l].A.n;
            info[4 * l + 1] = h.L[l].A.nnz;
            info[4 * l + 2] = (l + 1 < h.nlev) ? h.L[l].P.nnz : 0;
            info[4 * l + 3] = h.dense;
        }
        return CPTR_OK;
    });
}

cptr_status cptr_hierarchy_level(cptr_ctx *ctx, int32_t which, int32_t l, int32_t *rp, int32_t *ci, double *v,
                                 double *dinv, int32_t *cf, int32_t *Prp, int32_t *Pci, double *Pv) {
    return guarded(ctx, [&](Ctx *c) {
        CPTR_TRY(need_ready(c));
        const Hier &h = which == 0 ? c->hp : c->hT;
        if (which < 0 || which > 1 || l < 0 || l >= h.nlev) return c->fail(CPTR_EINVAL, "no such level");
        const Level &L = h.L[l];
        auto cp = [&](void *dst, const void *src, size_t bytes) -> cptr_status {
            if (dst && src && bytes) CPTR_TRY(copy_to_host(c, dst, src, bytes));
            return CPTR_OK;
        };
        CPTR_TRY(cp(rp, L.A.rp, sizeof(int32_t) * ((size_t)L.A.n + 1)));
        CPTR_TRY(cp(ci, L.A.ci, sizeof(int32_t) * (size_t)L.A.nnz));
        CPTR_TRY(cp(v, L.A.v, sizeof(double) * (size_t)L.A.nnz));
        CPTR_TRY(cp(dinv, L.dinv, sizeof(double) * (size_t)L.A.n));
        if (l + 1 < h.nlev) {
            CPTR_TRY(cp(cf, L.cf, sizeof(int32_t) * (size_t)L.A.n));
            CPTR_TRY(cp(Prp, L.P.rp, sizeof(int32_t) * ((size_t)L.A.n + 1)));
            CPTR_TRY(cp(Pci, L.P.ci, sizeof(int32_t) * (size_t)L.P.nnz));
            CPTR_TRY(cp(Pv, L.P.v, sizeof(double) * (size_t)L.P.nnz));
        }
        return CPTR_OK;
    });
}

int64_t cptr_launch_count(void) { return launch_count(); }

cptr_status cptr_inject_wait_timeout(cptr_ctx *ctx, int32_t on) {
    return guarded(ctx, [&](Ctx *c) {
        c->inject_wait = on ? 1 : 0;
        return CPTR_OK;
    });
}

cptr_status cptr_set_profiling(cptr_ctx *ctx, uint32_t mask) {
    return guarded(ctx, [&](Ctx *c) {
        c->prof.mask = mask;
        return CPTR_OK;
    });
}

cptr_status cptr_profile(cptr_ctx *ctx, double *ms, int64_t *count) {
    return guarded(ctx, [&](Ctx *c) {
        for (int f = 0; f < 16; ++f) {
            double m = 0.0;
            int64_t n = 0;
            if (f < PF_FAMILIES) { m = c->prof.ms[f]; n = c->prof.cnt[f]; }
            else { m = c->prof.setup_ms[f - PF_FAMILIES]; n = 1; }
            if (ms) ms[f] = m;
            if (count) count[f] = n;
        }
        return CPTR_OK;
    });
}

cptr_status cptr_profile_vcycle(cptr_ctx *ctx, double *ms, int64_t *count) {
    return guarded(ctx, [&](Ctx *c) {
        for (int k = 0; k < 8; ++k) {
            if (ms) ms[k] = c->prof.ms[PF_VC + k];
            if (count) count[k] = c->prof.cnt[PF_VC + k];
        }
        return CPTR_OK;
    });
}

cptr_status cptr_set_partition(cptr_ctx *ctx, int32_t n_cells, const int32_t *part, int32_t on_device) {
    return guarded(ctx, [&](Ctx *c) {
        dfree(c->part);
        c->part = nullptr;
        c->n_part = 0;
        ilu_sym_free(c);   // the ILU pattern changes with the partition
        if (!part) return CPTR_OK;
        if (n_cells <= 0) return c->fail(CPTR_EINVAL, "n_cells must be positive");
        CPTR_TRY(dalloc_t(c, &c->part, (size_t)n_cells));
        if (!host_or_device_copy(c, c->part, part, sizeof(int32_t) * (size_t)n_cells, on_device, cudaMemcpyHostToDevice))
            return c->fail(CPTR_ECUDA, "copy of the partition failed");
        CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        c->n_part = n_cells;
        return CPTR_OK;
    });
}

cptr_status cptr_tuning(cptr_ctx *ctx, int32_t *rows, int32_t cap, int32_t *n_rows) {
    return guarded(ctx, [&](Ctx *c) {
        CPTR_TRY(need_ready(c));
        if (!n_rows || (cap > 0 && !rows)) return c->fail(CPTR_EINVAL, "bad arguments");
        std::vector<int32_t> out;
        auto add = [&](int h, int l, int k, const Shape &sh) {
            for (int32_t v : {h, l, k, (int32_t)sh.G, (int32_t)sh.T}) out.push_back(v);
        };
        for (int h = 0; h < 2; ++h) {
            const Hier &H = h == 0 ? c->hp : c->hT;
            for (int l = 0; l + 1 < H.nlev; ++l) {
                add(h, l, 0, H.L[l].sh_A);
                add(h, l, 1, H.L[l].sh_PT);
                add(h, l, 2, H.L[l].sh_P);
            }
        }
        add(2, 0, 3, c->sell_shape);
        Shape isw;
        isw.G = (int16_t)c->sf_sleep;
        isw.T = (int16_t)c->sf_grid;
        add(3, 0, 4, isw);
        Shape chosen;
        chosen.G = c->tl_use ? 3 : (c->cw_use ? 1 : (c->sp_use ? 2 : 0));
        chosen.T = (int16_t)(c->sp_use ? c->sp_group : 0);
        add(3, 0, 5, chosen);
        Shape tile;
        tile.G = (int16_t)c->tl_best_ty;
        tile.T = (int16_t)c->tl_best_tz;
        add(3, 0, 6, tile);
        Shape lanes;
        lanes.G = (int16_t)(c->sp_use ? 4 * c->sf_half : 0);
        lanes.T = 0;
        add(3, 0, 7, lanes);
        *n_rows = (int32_t)(out.size() / 5);
        for (int32_t i = 0; i < std::min<int32_t>(cap, *n_rows) * 5; ++i) rows[i] = out[i];
        return CPTR_OK;
    });
}

cptr_status cptr_ilu_levels(cptr_ctx *ctx, int32_t *n_forward, int32_t *n_backward) {
    return guarded(ctx, [&](Ctx *c) {
        CPTR_TRY(need_ready(c));
        if (n_forward) *n_forward = c->nlev_f;
        if (n_backward) *n_backward = c->nlev_b;
        return CPTR_OK;
    });
}

}  // extern "C"

// ---- ensemble --------------------------------------------------------------------------------
namespace {
__global__ void k_copy_add(int32_t *dst, const int32_t *src, int64_t count, int32_t add) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = src[i] + add;
}

constexpr int64_t kTile = 8192;   // union-vector elements per Krylov tile

cptr_status batch_setup(Ctx *c, int32_t ni, int32_t b, const cptr_instance *inst, const int32_t *kind,
                        int on_device) {
    if (ni < 1 || !inst || !kind) return c->fail(CPTR_EINVAL, "n_inst >= 1, inst and unknown_kind are required");
    if (b != 3 && b != 4) return c->fail(CPTR_EINVAL, "b must be 3 or 4");
    const bool hasW = inst[0].row_weights != nullptr, hasS = inst[0].st_vals != nullptr;
    std::vector<int32_t> cell0(ni + 1, 0), nnz0(ni + 1, 0);
    for (int k = 0; k < ni; ++k) {
        const cptr_instance &I = inst[k];
        if (I.n_cells <= 0 || !I.row_ptr || !I.col_idx || !I.vals)
            return c->fail(CPTR_EINVAL, "instance " + std::to_string(k) + ": n_cells > 0 and the BSR arrays are required");
        if ((I.row_weights != nullptr) != hasW || (I.st_vals != nullptr) != hasS)
            return c->fail(CPTR_EINVAL, "row_weights and st_vals must be given for all instances or for none");
        int32_t nz = 0;
        if (on_device) CPTR_TRY(copy_to_host(c, &nz, I.row_ptr + I.n_cells, sizeof(int32_t)));
        else nz = I.row_ptr[I.n_cells];
        if (nz <= 0) return c->fail(CPTR_EINVAL, "instance " + std::to_string(k) + ": empty pattern");
        if ((int64_t)cell0[k] + I.n_cells > INT32_MAX || (int64_t)nnz0[k] + nz > INT32_MAX)
            return c->fail(CPTR_EINVAL, "the ensemble exceeds 2^31 cells or blocks");
        cell0[k + 1] = cell0[k] + I.n_cells;
        nnz0[k + 1] = nnz0[k] + nz;
    }
    const int32_t N = cell0[ni], NZ = nnz0[ni];
    const size_t bb = (size_t)b * b;
    int32_t *rp = nullptr, *ci = nullptr;
    double *vals = nullptr, *W = nullptr, *st = nullptr;
    struct Tmp {
        std::vector<void *> p;
        ~Tmp() { for (void *q : p) dfree(q); }
    } tmp;
    CPTR_TRY(dalloc_t(c, &rp, (size_t)N + 1)); tmp.p.push_back(rp);
    CPTR_TRY(dalloc_t(c, &ci, (size_t)NZ)); tmp.p.push_back(ci);
    CPTR_TRY(dalloc_t(c, &vals, (size_t)NZ * bb)); tmp.p.push_back(vals);
    if (hasW) { CPTR_TRY(dalloc_t(c, &W, (size_t)N * bb)); tmp.p.push_back(W); }
    if (hasS) { CPTR_TRY(dalloc_t(c, &st, (size_t)NZ)); tmp.p.push_back(st); }
    const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    int32_t *stage = nullptr;   // host pattern arrays are staged on the device before the offset
    int64_t stage_len = 0;
    for (int k = 0; k < ni; ++k) {
        const cptr_instance &I = inst[k];
        const int64_t nk = I.n_cells, zk = nnz0[k + 1] - nnz0[k];
        const int32_t *src_rp = I.row_ptr, *src_ci = I.col_idx;
        if (!on_device) {
            if (stage_len < nk + zk) {
                dfree(stage);
                stage = nullptr;
                CPTR_TRY(dalloc_t(c, &stage, (size_t)(nk + zk)));
                stage_len = nk + zk;
            }
            CPTR_CUDA_TRY(c, cudaMemcpyAsync(stage, I.row_ptr, sizeof(int32_t) * nk, cudaMemcpyHostToDevice, c->stream));
            CPTR_CUDA_TRY(c, cudaMemcpyAsync(stage + nk, I.col_idx, sizeof(int32_t) * zk, cudaMemcpyHostToDevice,
                                             c->stream));
            src_rp = stage;
            src_ci = stage + nk;
        }
        (k_copy_add<<<(unsigned)((nk + 255) / 256), 256, 0, c->stream>>>(rp + cell0[k], src_rp, nk, nnz0[k]),
         note_launch());
        (k_copy_add<<<(unsigned)((zk + 255) / 256), 256, 0, c->stream>>>(ci + nnz0[k], src_ci, zk, cell0[k]),
         note_launch());
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(vals + (size_t)nnz0[k] * bb, I.vals, sizeof(double) * zk * bb, kin, c->stream));
        if (hasW)
            CPTR_CUDA_TRY(c, cudaMemcpyAsync(W + (size_t)cell0[k] * bb, I.row_weights, sizeof(double) * nk * bb, kin,
                                             c->stream));
        if (hasS)
            CPTR_CUDA_TRY(c, cudaMemcpyAsync(st + nnz0[k], I.st_vals, sizeof(double) * zk, kin, c->stream));
        if (!on_device) CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));   // stage is reused
    }
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(rp + N, &NZ, sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    int32_t hk[4];
    if (on_device) CPTR_TRY(copy_to_host(c, hk, kind, sizeof(int32_t) * b));
    else memcpy(hk, kind, sizeof(int32_t) * b);
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    dfree(stage);
    CPTR_CUDA_TRY(c, cudaGetLastError());
    CPTR_TRY(do_setup(c, N, b, rp, ci, vals, hk, W, st, 1, 0));
    // tiles of the union vector, none straddling two instances
    std::vector<int32_t> t_inst, i_t0(ni + 1, 0);
    std::vector<int64_t> t_beg;
    for (int k = 0; k < ni; ++k) {
        i_t0[k] = (int32_t)t_inst.size();
        const int64_t beg = (int64_t)cell0[k] * b, end = (int64_t)cell0[k + 1] * b;
        for (int64_t p = beg; p < end; p += kTile) {
            t_inst.push_back(k);
            t_beg.push_back(p);
        }
    }
    i_t0[ni] = (int32_t)t_inst.size();
    t_beg.push_back((int64_t)N * b);
    c->n_tiles = (int32_t)t_inst.size();
    CPTR_TRY(dalloc_t(c, &c->tile_inst, t_inst.size()));
    CPTR_TRY(dalloc_t(c, &c->tile_beg, t_beg.size()));
    CPTR_TRY(dalloc_t(c, &c->inst_tile0, i_t0.size()));
    CPTR_TRY(dalloc_t(c, &c->ksb, (size_t)ni));
    CPTR_TRY(dalloc_t(c, &c->hdr, (size_t)ni + 1));
    CPTR_TRY(dalloc_t(c, &c->partial_b, (size_t)c->n_tiles * (kMaxRestart + 1)));
    CPTR_CUDA_TRY(c, cudaMallocHost((void **)&c->hdr_host, sizeof(KHdr) * (ni + 1)));
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->tile_inst, t_inst.data(), sizeof(int32_t) * t_inst.size(), cudaMemcpyHostToDevice, c->stream));
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->tile_beg, t_beg.data(), sizeof(int64_t) * t_beg.size(), cudaMemcpyHostToDevice, c->stream));
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->inst_tile0, i_t0.data(), sizeof(int32_t) * i_t0.size(), cudaMemcpyHostToDevice, c->stream));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(c->ksb, 0, sizeof(KState) * ni, c->stream));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(c->vcur, 0, sizeof(double) * N * b, c->stream));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(c->zcur, 0, sizeof(double) * N * b, c->stream));
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->n_inst = ni;
    c->inst_cell0 = cell0;
    return CPTR_OK;
}
}  // namespace

extern "C" {
cptr_status cptr_setup_batch(cptr_ctx *ctx, int32_t n_inst, int32_t b, const cptr_instance *inst,
                             const int32_t *unknown_kind, int32_t on_device) {
    return guarded(ctx, [&](Ctx *c) {
        cptr_status s = batch_setup(c, n_inst, b, inst, unknown_kind, on_device);
        if (s != CPTR_OK) {
            std::string keep = c->err;
            cudaStreamSynchronize(c->stream);
            release_setup(c);
            c->err = keep;
        }
        return s;
    });
}

cptr_status cptr_solve_batch(cptr_ctx *ctx, const double *const *rhs, double *const *x, double rtol, cptr_stats *st,
                             int32_t on_device) {
    return guarded(ctx, [&](Ctx *c) {
        CPTR_TRY(need_ready(c));
        if (c->n_inst < 1) return c->fail(CPTR_ESTATE, "the last set-up was not cptr_setup_batch");
        if (!rhs || !x) return c->fail(CPTR_EINVAL, "rhs and x are required");
        if (!(rtol >= 0.0)) return c->fail(CPTR_EINVAL, "rtol must be >= 0");
        const int ni = c->n_inst, b = c->b;
        for (int k = 0; k < ni; ++k)
            if (!rhs[k] || !x[k]) return c->fail(CPTR_EINVAL, "rhs[k] and x[k] are required for every instance");
        cudaEvent_t e0, e1;
        CPTR_CUDA_TRY(c, cudaEventCreate(&e0));
        CPTR_CUDA_TRY(c, cudaEventCreate(&e1));
        CPTR_CUDA_TRY(c, cudaEventRecord(e0, c->stream));
        const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        const cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        for (int k = 0; k < ni; ++k) {
            const size_t off = (size_t)c->inst_cell0[k] * b, len = (size_t)(c->inst_cell0[k + 1] - c->inst_cell0[k]) * b;
            CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->xw + off, rhs[k], sizeof(double) * len, kin, c->stream));
        }
        launch_weight_vec(c, c->W, c->xw, c->bw);
        prof_reset(c);
        cptr_status s = fgmres_solve_batch(c, c->bw, c->xw, rtol, st);
        if (s == CPTR_OK || s == CPTR_NOT_CONVERGED)
            for (int k = 0; k < ni; ++k) {
                const size_t off = (size_t)c->inst_cell0[k] * b, len = (size_t)(c->inst_cell0[k + 1] - c->inst_cell0[k]) * b;
                CPTR_CUDA_TRY(c, cudaMemcpyAsync(x[k], c->xw + off, sizeof(double) * len, kout, c->stream));
            }
        CPTR_CUDA_TRY(c, cudaEventRecord(e1, c->stream));
        CPTR_CUDA_TRY(c, cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (st)
            for (int k = 0; k < ni; ++k) {
                st[k].solve_ms = ms;
                st[k].setup_ms = c->setup_ms;
                st[k].levels_p = c->hp.nlev;
                st[k].levels_T = c->hT.nlev;
                st[k].op_complexity_p = c->hp.op_complexity;
                st[k].op_complexity_T = c->hT.op_complexity;
                st[k].schur_used = c->schur_used;
            }
        return s;
    });
}
}  // extern "C"

extern "C" {

// ---- learned Schur scaling ----------------------------------------------------------------------

cptr_status cptr_schur_features(cptr_ctx *ctx, double *feat, int32_t on_device) {
    return guarded(ctx, [&](Ctx *c) {
        CPTR_TRY(need_ready(c));
        if (!feat) return c->fail(CPTR_EINVAL, "feat is required");
        DevOut<double> out;
        CPTR_TRY(out.init(c, feat, (size_t)c->n * CPTR_MLP_FEATURES, on_device));
        CPTR_TRY(learned_features(c, out.p));
        return out.finish(c);
    });
}

cptr_status cptr_mlp_loss_grad(cptr_ctx *ctx, const double *feat, const double *target, int32_t n,
                               const float *params, float *grad, double *loss, int32_t on_device) {
    return guarded(ctx, [&](Ctx *c) {
        if (n < 1 || !feat || !target || !params || !grad) return c->fail(CPTR_EINVAL, "bad arguments");
        DevIn<double> f, t;
        DevIn<float> P;
        DevOut<float> g;
        CPTR_TRY(f.init(c, feat, (size_t)n * CPTR_MLP_FEATURES, on_device));
        CPTR_TRY(t.init(c, target, (size_t)n, on_device));
        CPTR_TRY(P.init(c, params, CPTR_MLP_NPARAM, on_device));
        CPTR_TRY(g.init(c, grad, CPTR_MLP_NPARAM, on_device));
        CPTR_TRY(mlp_loss_grad(c, f.p, t.p, n, P.p, g.p, loss));
        return g.finish(c);
    });
}

cptr_status cptr_mlp_train(cptr_ctx *ctx, const double *feat, const double *target, int32_t n, float *params,
                           int32_t steps, float lr, double *loss_hist, int32_t on_device) {
    return guarded(ctx, [&](Ctx *c) {
        if (n < 1 || steps < 0 || !feat || !target || !params || !(lr > 0.f))
            return c->fail(CPTR_EINVAL, "bad arguments");
        DevIn<double> f, t;
        DevOut<float> P;
        CPTR_TRY(f.init(c, feat, (size_t)n * CPTR_MLP_FEATURES, on_device));
        CPTR_TRY(t.init(c, target, (size_t)n, on_device));
        CPTR_TRY(P.init(c, params, CPTR_MLP_NPARAM, on_device));
        if (!on_device)
            CPTR_CUDA_TRY(c, cudaMemcpyAsync(P.p, params, sizeof(float) * CPTR_MLP_NPARAM, cudaMemcpyHostToDevice,
                                             c->stream));
        CPTR_TRY(mlp_train(c, f.p, t.p, n, P.p, steps, lr, loss_hist));
        return P.finish(c);
    });
}

cptr_status cptr_set_mlp(cptr_ctx *ctx, const float *params, int32_t on_device) {
    return guarded(ctx, [&](Ctx *c) {
        if (!params) {
            dfree(c->mlp);
            c->mlp = nullptr;
            return sync(c);
        }
        if (!c->mlp) CPTR_TRY(dalloc_t(c, &c->mlp, CPTR_MLP_NPARAM));
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(c->mlp, params, sizeof(float) * CPTR_MLP_NPARAM,
                                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
        return sync(c);
    });
}

cptr_status cptr_mlp_infer(cptr_ctx *ctx, const double *feat, int32_t n, float *y, int32_t on_device) {
    return guarded(ctx, [&](Ctx *c) {
        if (!c->mlp) return c->fail(CPTR_ESTATE, "no network (cptr_set_mlp)");
        if (n < 1 || !feat || !y) return c->fail(CPTR_EINVAL, "bad arguments");
        DevIn<double> f;
        DevOut<float> out;
        CPTR_TRY(f.init(c, feat, (size_t)n * CPTR_MLP_FEATURES, on_device));
        CPTR_TRY(out.init(c, y, (size_t)n, on_device));
        CPTR_TRY(mlp_infer(c, f.p, n, out.p));
        return out.finish(c);
    });
}

cptr_status cptr_schur_scaling(cptr_ctx *ctx, double *s, int32_t on_device) {
    return guarded(ctx, [&](Ctx *c) {
        CPTR_TRY(need_ready(c));
        if (!s) return c->fail(CPTR_EINVAL, "s is required");
        if (c->schur_used == CPTR_SCHUR_LEARNED && c->lf_s) {
            if (on_device)
                CPTR_CUDA_TRY(c, cudaMemcpyAsync(s, c->lf_s, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, c->stream));
            else
                return copy_to_host(c, s, c->lf_s, sizeof(double) * c->n);
            return sync(c);
        }
        if (on_device) {
            std::vector<double> ones((size_t)c->n, 1.0);
            CPTR_CUDA_TRY(c, cudaMemcpyAsync(s, ones.data(), sizeof(double) * c->n, cudaMemcpyHostToDevice, c->stream));
            return sync(c);
        }
        for (int32_t i = 0; i < c->n; ++i) s[i] = 1.0;
        return CPTR_OK;
    });
}

}  // extern "C"
