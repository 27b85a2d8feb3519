// Device-side synchronisation primitives of the one-launch triangular sweeps (ilu.cu,
// ilu_tile.cu).  The values of an unsolved row hold a sentinel NaN payload that arithmetic never
// produces; a producer publishes a value with a relaxed GPU-scope store and a consumer polls it
// with relaxed GPU-scope loads, so every value doubles as its own ready flag.  Every wait is
// bounded by kWaitNs of GPU time; a wait that gives up sets ks->wait_err and the call reports
// CPTR_ETIMEOUT.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace cptr {

constexpr unsigned long long kSentinel = 0x7FF4C0DEDEADBEEFULL;  // never produced by arithmetic
constexpr unsigned kSentinel32 = 0x7FA6C0DEu;                      // the same for FP32 vectors
constexpr unsigned long long kWaitNs = 500ULL * 1000ULL * 1000ULL;
constexpr int kSfThreads = 128;

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// loads and stores the compiler may neither hoist out of a loop nor merge (relaxed, GPU scope:
// they observe / publish values through L2 for other SMs)
__device__ __forceinline__ double load_relaxed(const double *p) {
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ float load_relaxed(const float *p) {
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void store_relaxed(double *p, double v) {
    asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void store_relaxed(float *p, float v) {
    asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ double load_acquire(const double *p) {
    double v;
    asm volatile("ld.acquire.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ bool is_sentinel(double v) { return __double_as_longlong(v) == (long long)kSentinel; }
__device__ __forceinline__ bool is_sentinel(float v) { return __float_as_uint(v) == kSentinel32; }
template <typename T> __device__ __forceinline__ T sentinel_value();
template <> __device__ __forceinline__ double sentinel_value<double>() { return __longlong_as_double((long long)kSentinel); }
template <> __device__ __forceinline__ float sentinel_value<float>() { return __uint_as_float(kSentinel32); }

// wait (bounded) until *p no longer holds the sentinel; returns its value (failure injection)
__device__ __forceinline__ double wait_value(const double *p, KState *ks) {
    double v = load_acquire(p);
    if (!is_sentinel(v)) return v;
    const unsigned long long t0 = gtimer();
    for (;;) {
        __nanosleep(40);
        v = load_acquire(p);
        if (!is_sentinel(v)) return v;
        if (gtimer() - t0 > kWaitNs) {
            atomicExch(&ks->wait_err, 1);
            return 0.0;
        }
    }
}


}  // namespace cptr
