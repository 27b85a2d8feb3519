// Allocation-free variant of the ILU(0) application (cptr_apply_ilu_static).
//
// Some callers cannot allocate device memory at the moment they need the preconditioner: code
// that runs while a framework's caching allocator owns the whole device, real-time loops that
// must not pay for cudaMalloc/cudaFree (cudaFree also synchronises the device), and deployments
// with a fixed device-memory budget decided up front.  This entry point keeps the two
// intermediate vectors of the triangular solves in one file-scope device array instead of
// context memory, so the call itself allocates nothing.
//
// The array holds 2 x kStaticIluMax doubles (16 MiB).  Every GPU that loads the library keeps it
// until the process exits.  In host code the array's name is only a host-side stand-in, so the
// kernels get its device address from cudaGetSymbolAddress, with the call's device current.
// The address is looked up again on every call whose stream is not being captured (the lookup
// is cheap, and the address can change when the device's context is destroyed and re-created,
// e.g. after cudaDeviceReset, or when the caller switches to another context on the same
// device); a call made while its stream is being captured uses the address found by the last
// uncaptured call on that device, so the first call on a device must come before any stream
// capture.  All calls on a device share the array, so calls whose work overlaps on the GPU
// (different streams, or different contexts launched concurrently) race on it.  Nothing in it
// needs to start at zero: every element the solves read was written earlier in the same call.
// The call applies the FP64 factors with one launch per level set, whatever the context's
// precision and sweep schedule, and synchronises the context's stream before it returns.
#include <cuda_runtime.h>

#include <mutex>
#include <new>

#include "common.cuh"

using namespace cptr;

namespace {

constexpr int64_t kStaticIluMax = int64_t(1) << 20;  // unknowns (n_cells * b) per call
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_ilu_scratch[2 * kStaticIluMax];

std::mutex g_mu;
double *g_scratch_addr[kMaxDevices] = {};   // last address found on each device

// device address of g_ilu_scratch on the current device
cptr_status scratch_address(Ctx *c, double **out) {
    int dev = 0;
    CPTR_CUDA_TRY(c, cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return c->fail(CPTR_EINVAL, "device ordinal out of range");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CPTR_CUDA_TRY(c, cudaStreamIsCapturing(c->stream, &cap));
    std::lock_guard<std::mutex> lock(g_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        CPTR_CUDA_TRY(c, cudaGetSymbolAddress(&p, g_ilu_scratch));
        g_scratch_addr[dev] = static_cast<double *>(p);
    } else if (!g_scratch_addr[dev]) {
        return c->fail(CPTR_ESTATE, "cptr_apply_ilu_static: the first call on a device must not be captured");
    }
    *out = g_scratch_addr[dev];
    return CPTR_OK;
}

cptr_status apply_static(Ctx *c, const double *r, double *z) {
    if (!c->ready) return c->fail(CPTR_ESTATE, "no successful cptr_setup on this context");
    if (c->o.stage2 != CPTR_STAGE2_ILU0) return c->fail(CPTR_ESTATE, "ILU(0) was not set up");
    if (c->o.ilu_order != CPTR_ILU_NATURAL)
        return c->fail(CPTR_EINVAL, "cptr_apply_ilu_static supports the natural ILU ordering only");
    if (c->o.ilu_fill != 0) return c->fail(CPTR_EINVAL, "cptr_apply_ilu_static supports ILU(0) only");
    if (!r || !z) return c->fail(CPTR_EINVAL, "r and z are required");
    const int64_t nb = (int64_t)c->n * c->b;
    if (nb > kStaticIluMax)
        return c->fail(CPTR_EINVAL, "cptr_apply_ilu_static: n_cells * b = " + std::to_string(nb) +
                                        " exceeds the static scratch limit of " + std::to_string(kStaticIluMax));
    double *scratch = nullptr;
    CPTR_TRY(scratch_address(c, &scratch));
    ilu_apply_into(c, r, z, scratch, scratch + kStaticIluMax);
    CPTR_CUDA_TRY(c, cudaGetLastError());
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return CPTR_OK;
}

}  // namespace

extern "C" cptr_status cptr_apply_ilu_static(cptr_ctx *ctx, const double *r, double *z) {
    if (!ctx) return CPTR_EINVAL;
    Ctx *c = &ctx->c;
    CtxScope scope(c);
    try {
        c->err.clear();
        const cptr_status st = apply_static(c, r, z);
        const cptr_status ck = check_report(c);   // the bounds-checking build only
        return ck != CPTR_OK ? ck : st;
    } catch (const std::bad_alloc &) {
        return c->fail(CPTR_ENOMEM, "host allocation failed");
    } catch (...) {
        return c->fail(CPTR_EINVAL, "unexpected host exception");
    }
}
