// Learned diagonal scaling of the temperature Schur approximation.  The paper approximates
// S_T = A_TT - A_Tp A_pp^{-1} A_pT by the discrete S_e or, without it, by A_TT (Sec. 3.3.1); this
// extension scales the rows of that base approximation B, S~_T = diag(s) B, s_i = sinh(y_i), y_i
// the output of a 16-64-64-1 tanh network over local features of cell i of A'.
//
//   k_sat_terms        per-cell saturation terms of features 7 and 8 (from the BSR A', set-up)
//   k_learned_schur    features + BF16 inference + row scaling, one thread per cell, fused
//   k_features         features only (for training data)
//   k_infer            BF16 inference on given features
//   k_mlp_grad         FP32 forward + backward over 64-sample tiles, per-CTA partial gradients
//   k_mlp_reduce       ordered reduction of the partials (+ one Adam step, or the raw gradient)
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace cptr {
namespace {

constexpr int NF = CPTR_MLP_FEATURES, NH = CPTR_MLP_HIDDEN;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NF, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH, NPARAM = OFF_B3 + 1;
static_assert(NPARAM == CPTR_MLP_NPARAM, "parameter layout");
constexpr float kMaxAbsY = 30.0f;   // larger outputs (|s| > 5e12) reject the network's scaling

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ double qdiv(double x, double y) { return y == 0.0 ? 0.0 : x / y; }
__device__ __forceinline__ double sgn(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// ---- features --------------------------------------------------------------------------------
struct FeatIn {
    const int32_t *rp, *ci, *diag;
    const double *App, *ApT, *ATp, *B, *sat;   // B: the base approximation
};

__global__ void k_sat_terms(int32_t n, int b, int ps, int ts, const int32_t *diag, const double *A, double *sat) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *a = A + (int64_t)diag[i] * b * b;
    double s7 = 0.0, s8 = 0.0;
    for (int s = 0; s < b; ++s) {
        if (s == ps || s == ts) continue;
        double ass = a[s * b + s];
        s7 = __dadd_rn(s7, __dmul_rn(a[ts * b + s], qdiv(a[s * b + ts], ass)));
        s8 = __dadd_rn(s8, __dmul_rn(a[ps * b + s], qdiv(a[s * b + ps], ass)));
    }
    sat[2 * i] = s7;
    sat[2 * i + 1] = s8;
}

// value of a cell-pattern field at (row, col), 0 if the pattern has no such entry
__device__ __forceinline__ double field_at(const FeatIn &in, const double *F, int32_t row, int32_t col) {
    for (int32_t k = in.rp[row]; k < in.rp[row + 1]; ++k)
        if (in.ci[k] == col) return F[k];
    return 0.0;
}

// the 16 features of cell i (already through asinh); sums in ascending pattern order with
// separately rounded products and sums
__device__ void cell_features(const FeatIn &in, int32_t i, double f[NF]) {
    const int32_t k0 = in.rp[i], k1 = in.rp[i + 1], d = in.diag[i];
    const double app = in.App[d], bii = in.B[d], apt = in.ApT[d], atp = in.ATp[d];
    double s0 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0, s6 = 0, s14 = 0, s15 = 0;
    for (int32_t k = k0; k < k1; ++k) {
        const int32_t j = in.ci[k];
        const double t = __dmul_rn(in.ATp[k], qdiv(field_at(in, in.ApT, j, i), in.App[in.diag[j]]));
        s0 = __dadd_rn(s0, t);
        s6 = __dadd_rn(s6, fabs(t));
        if (j != i) {
            s2 = __dadd_rn(s2, fabs(in.App[k]));
            s3 = __dadd_rn(s3, fabs(in.B[k]));
            s4 = __dadd_rn(s4, in.App[k]);
            s5 = __dadd_rn(s5, in.B[k]);
            s14 = __dadd_rn(s14, fabs(in.ApT[k]));
            s15 = __dadd_rn(s15, fabs(in.ATp[k]));
        }
    }
    const double pb = fabs(__dmul_rn(app, bii)), r = sqrt(pb);
    f[0] = qdiv(s0, bii);
    f[1] = qdiv(__dmul_rn(atp, qdiv(apt, app)), bii);
    f[2] = qdiv(s2, fabs(app));
    f[3] = qdiv(s3, fabs(bii));
    f[4] = qdiv(s4, fabs(app));
    f[5] = qdiv(s5, fabs(bii));
    f[6] = qdiv(s6, fabs(bii));
    f[7] = qdiv(in.sat[2 * i], bii);
    f[8] = qdiv(in.sat[2 * i + 1], app);
    f[9] = sgn(app);
    f[10] = sgn(bii);
    f[11] = qdiv(apt, r);
    f[12] = qdiv(atp, r);
    f[13] = (double)(k1 - k0) / 7.0;
    f[14] = qdiv(__dmul_rn(s14, fabs(atp)), pb);
    f[15] = qdiv(__dmul_rn(s15, fabs(apt)), pb);
#pragma unroll
    for (int q = 0; q < NF; ++q) f[q] = asinh(f[q]);
}

// ---- BF16 inference ---------------------------------------------------------------------------
// Weights rounded to BF16 once per block (held as floats in shared memory), biases FP32.
struct InferW {
    float w1t[NF * NH];   // w1t[q][j] = W1[j][q]
    float w2[NH * NH];
    float w3[NH];
    float b1[NH], b2[NH];
    float b3;
};

__device__ void load_infer_weights(InferW &W, const float *P) {
    for (int q = threadIdx.x; q < NH * NF; q += blockDim.x) W.w1t[(q % NF) * NH + q / NF] = bf16r(P[OFF_W1 + q]);
    for (int q = threadIdx.x; q < NH * NH; q += blockDim.x) W.w2[q] = bf16r(P[OFF_W2 + q]);
    for (int q = threadIdx.x; q < NH; q += blockDim.x) {
        W.w3[q] = bf16r(P[OFF_W3 + q]);
        W.b1[q] = P[OFF_B1 + q];
        W.b2[q] = P[OFF_B2 + q];
    }
    if (threadIdx.x == 0) W.b3 = P[OFF_B3];
    __syncthreads();
}

// y = w3 . h2 + b3 with h1, h2 rounded to BF16; every sum starts at the bias and adds the exact
// BF16 x BF16 products in ascending input order, rounding to FP32 after each addition
__device__ float infer_cell(const InferW &W, const float x[NF]) {
    float h1[NH];
#pragma unroll
    for (int j = 0; j < NH; ++j) h1[j] = W.b1[j];
#pragma unroll
    for (int q = 0; q < NF; ++q) {
        const float4 *col = reinterpret_cast<const float4 *>(W.w1t + q * NH);
#pragma unroll
        for (int j4 = 0; j4 < NH / 4; ++j4) {
            const float4 w = col[j4];
            h1[4 * j4 + 0] = fmaf(w.x, x[q], h1[4 * j4 + 0]);
            h1[4 * j4 + 1] = fmaf(w.y, x[q], h1[4 * j4 + 1]);
            h1[4 * j4 + 2] = fmaf(w.z, x[q], h1[4 * j4 + 2]);
            h1[4 * j4 + 3] = fmaf(w.w, x[q], h1[4 * j4 + 3]);
        }
    }
#pragma unroll
    for (int j = 0; j < NH; ++j) h1[j] = bf16r(tanhf(h1[j]));
    float out = W.b3;
#pragma unroll 1
    for (int j = 0; j < NH; ++j) {
        const float4 *row = reinterpret_cast<const float4 *>(W.w2 + j * NH);
        float acc = W.b2[j];
#pragma unroll
        for (int q = 0; q < NH / 4; ++q) {
            const float4 w = row[q];
            acc = fmaf(w.x, h1[4 * q + 0], acc);
            acc = fmaf(w.y, h1[4 * q + 1], acc);
            acc = fmaf(w.z, h1[4 * q + 2], acc);
            acc = fmaf(w.w, h1[4 * q + 3], acc);
        }
        out = fmaf(W.w3[j], bf16r(tanhf(acc)), out);
    }
    return out;
}

// features (FP64) -> network inputs: FP32 then BF16, both round to nearest even
__device__ __forceinline__ void to_inputs(const double f[NF], float x[NF]) {
#pragma unroll
    for (int q = 0; q < NF; ++q) x[q] = bf16r((float)f[q]);
}

// S~_T = diag(s) B with s_i = sinh(y_i); flag = 1 if any s is unusable
__global__ void __launch_bounds__(256) k_learned_schur(FeatIn in, int32_t n, const float *P, double *St, double *s_out,
                                                       int32_t *flag) {
    __shared__ __align__(16) InferW W;
    load_infer_weights(W, P);
    // one cell per thread: a grid-stride loop would let the compiler hoist the (loop-invariant)
    // shared-memory weight loads into registers and spill
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        float x[NF];
        {
            double f[NF];
            cell_features(in, i, f);
            to_inputs(f, x);
        }
        const float y = infer_cell(W, x);
        const double s = sinh((double)y);
        if (!(fabsf(y) <= kMaxAbsY) || !isfinite(s)) atomicOr(flag, 1);
        s_out[i] = s;
        for (int32_t k = in.rp[i]; k < in.rp[i + 1]; ++k) St[k] = __dmul_rn(s, in.B[k]);
    }
}

__global__ void k_features(FeatIn in, int32_t n, double *feat) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double f[NF];
    cell_features(in, i, f);
#pragma unroll
    for (int q = 0; q < NF; ++q) feat[(int64_t)i * NF + q] = f[q];
}

__global__ void __launch_bounds__(256) k_infer(const double *feat, int32_t n, const float *P, float *y) {
    __shared__ __align__(16) InferW W;
    load_infer_weights(W, P);
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        double f[NF];
#pragma unroll
        for (int q = 0; q < NF; ++q) f[q] = feat[(int64_t)i * NF + q];
        float x[NF];
        to_inputs(f, x);
        y[i] = infer_cell(W, x);
    }
}

__global__ void k_fill(double *v, int32_t n, double a) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = a;
}

// ---- training (FP32) ----------------------------------------------------------------------------
// One CTA of 256 threads walks 64-sample tiles (tile blockIdx.x, + gridDim.x, ...).  Every
// parameter's gradient has one owning thread that accumulates it over the CTA's tiles in a fixed
// order; the partials of all CTAs are then summed in CTA order, so the result is deterministic.
constexpr int TS = 64, TT = 256, LD = NH + 1;
constexpr int kTrainCtas = 2 * 152;

struct TrainSmem {
    float w1t[NF * NH];   // w1t[k][j] = W1[j][k]
    float w2t[NH * NH];   // w2t[k][j] = W2[j][k]
    float w2[NH * NH];    // W2[j][k]
    float b1[NH], b2[NH], w3[NH];
    float x[TS * NF];
    float h1[TS * LD], h2[TS * LD], d2[TS * LD], d1[TS * LD];
    float dy[TS];
    float b3;
};

// out[s][j] = tanh(bias[j] + sum_k A[s][k] BT[k][j]) for a 64 x 64 tile; thread (ty, tx) owns
// samples 4ty..4ty+3 and units 4tx..4tx+3
template <int K>
__device__ __forceinline__ void tile_tanh(const float *A, int lda, const float *BT, const float *bias, float *out) {
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = bias[4 * tx + c];
#pragma unroll 8
    for (int k = 0; k < K; ++k) {
        const float4 bv = *reinterpret_cast<const float4 *>(BT + k * NH + 4 * tx);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const float av = A[(4 * ty + a) * lda + k];
            acc[a][0] = fmaf(av, bv.x, acc[a][0]);
            acc[a][1] = fmaf(av, bv.y, acc[a][1]);
            acc[a][2] = fmaf(av, bv.z, acc[a][2]);
            acc[a][3] = fmaf(av, bv.w, acc[a][3]);
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) out[(4 * ty + a) * LD + 4 * tx + c] = tanhf(acc[a][c]);
}

__global__ void __launch_bounds__(TT, 2) k_mlp_grad(const float *X, const float *T, int32_t n, const float *P,
                                                    float *part, double *loss_part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem &S = *reinterpret_cast<TrainSmem *>(smem_raw);
    const int t = threadIdx.x;
    for (int q = t; q < NH * NF; q += TT) {
        const int j = q / NF, k = q % NF;
        S.w1t[k * NH + j] = P[OFF_W1 + q];
    }
    for (int q = t; q < NH * NH; q += TT) {
        const int j = q / NH, k = q % NH;
        S.w2[q] = P[OFF_W2 + q];
        S.w2t[k * NH + j] = P[OFF_W2 + q];
    }
    if (t < NH) {
        S.b1[t] = P[OFF_B1 + t];
        S.b2[t] = P[OFF_B2 + t];
        S.w3[t] = P[OFF_W3 + t];
    }
    if (t == 0) S.b3 = P[OFF_B3];
    // owned gradients
    const int ty = t >> 4, tx = t & 15;
    float gW2[4][4] = {};
    float gW1[4] = {};
    float gvec = 0.f;   // b2 (t < 64), w3 (64 <= t < 128), b1 (128 <= t < 192), b3 (t == 192)
    double lsum = 0.0;
    const float inv_n = 1.0f / (float)n;
    const int ntiles = (n + TS - 1) / TS;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t base = (int64_t)tile * TS;
        __syncthreads();   // previous tile fully consumed (and weights loaded)
        for (int q = t; q < TS * NF; q += TT) {
            const int64_t s = base + q / NF;
            S.x[q] = s < n ? X[base * NF + q] : 0.f;
        }
        __syncthreads();
        tile_tanh<NF>(S.x, NF, S.w1t, S.b1, S.h1);
        __syncthreads();
        tile_tanh<NH>(S.h1, LD, S.w2t, S.b2, S.h2);
        __syncthreads();
        if (t < TS) {
            float y = S.b3;
            for (int j = 0; j < NH; ++j) y = fmaf(S.w3[j], S.h2[t * LD + j], y);
            const bool valid = base + t < n;
            const float e = valid ? y - T[base + t] : 0.f;
            S.dy[t] = 2.f * e * inv_n;
            lsum += (double)e * (double)e;
        }
        __syncthreads();
        for (int q = t; q < TS * NH; q += TT) {
            const int s = q / NH, j = q % NH;
            const float h = S.h2[s * LD + j];
            S.d2[s * LD + j] = S.dy[s] * S.w3[j] * (1.f - h * h);
        }
        __syncthreads();
        // dW2[j][k] += d2[s][j] h1[s][k]; b2, w3, b3
        for (int s = 0; s < TS; ++s) {
            float a[4], c[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = S.d2[s * LD + 4 * ty + q];
                c[q] = S.h1[s * LD + 4 * tx + q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) gW2[p][q] = fmaf(a[p], c[q], gW2[p][q]);
        }
        if (t < NH) {
            for (int s = 0; s < TS; ++s) gvec += S.d2[s * LD + t];
        } else if (t < 2 * NH) {
            for (int s = 0; s < TS; ++s) gvec = fmaf(S.dy[s], S.h2[s * LD + t - NH], gvec);
        } else if (t == 3 * NH) {
            for (int s = 0; s < TS; ++s) gvec += S.dy[s];
        }
        // d1 = (d2 W2) * (1 - h1^2)
        {
            float acc[4][4] = {};
#pragma unroll 8
            for (int j = 0; j < NH; ++j) {
                const float4 wv = *reinterpret_cast<const float4 *>(S.w2 + j * NH + 4 * tx);
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const float dv = S.d2[(4 * ty + a) * LD + j];
                    acc[a][0] = fmaf(dv, wv.x, acc[a][0]);
                    acc[a][1] = fmaf(dv, wv.y, acc[a][1]);
                    acc[a][2] = fmaf(dv, wv.z, acc[a][2]);
                    acc[a][3] = fmaf(dv, wv.w, acc[a][3]);
                }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int o = (4 * ty + a) * LD + 4 * tx + c;
                    const float h = S.h1[o];
                    S.d1[o] = acc[a][c] * (1.f - h * h);
                }
        }
        __syncthreads();
        // dW1[j][k] += d1[s][j] x[s][k] (thread: j = t / 4, k = 4 (t % 4) .. +3); b1
        {
            const int j = t >> 2, k0 = (t & 3) * 4;
            for (int s = 0; s < TS; ++s) {
                const float dv = S.d1[s * LD + j];
                const float4 xv = *reinterpret_cast<const float4 *>(S.x + s * NF + k0);
                gW1[0] = fmaf(dv, xv.x, gW1[0]);
                gW1[1] = fmaf(dv, xv.y, gW1[1]);
                gW1[2] = fmaf(dv, xv.z, gW1[2]);
                gW1[3] = fmaf(dv, xv.w, gW1[3]);
            }
            if (t >= 2 * NH && t < 3 * NH)
                for (int s = 0; s < TS; ++s) gvec += S.d1[s * LD + t - 2 * NH];
        }
    }
    // this CTA's partial gradient
    float *out = part + (int64_t)blockIdx.x * NPARAM;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) out[OFF_W2 + (4 * ty + p) * NH + 4 * tx + q] = gW2[p][q];
#pragma unroll
    for (int q = 0; q < 4; ++q) out[OFF_W1 + (t >> 2) * NF + (t & 3) * 4 + q] = gW1[q];
    if (t < NH) out[OFF_B2 + t] = gvec;
    else if (t < 2 * NH) out[OFF_W3 + t - NH] = gvec;
    else if (t < 3 * NH) out[OFF_B1 + t - 2 * NH] = gvec;
    else if (t == 3 * NH) out[OFF_B3] = gvec;
    // loss partial (threads 0..63 hold sample losses)
    double l = lsum;
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    __shared__ double lred[TT / 32];
    if ((t & 31) == 0) lred[t >> 5] = l;
    __syncthreads();
    if (t == 0) {
        double a = 0.0;
        for (int w = 0; w < TT / 32; ++w) a += lred[w];
        loss_part[blockIdx.x] = a;
    }
}

// g = sum over CTAs (ascending, FP64); then either grad = g, or one Adam step on P (FP32) with
// bias corrections c1 = 1 - beta1^t, c2 = 1 - beta2^t.  loss[0] = sum of loss partials / n.
__global__ void k_mlp_reduce(const float *part, const double *loss_part, int nparts, int32_t n, float *grad, float *P,
                             float *m, float *v, float lr, float c1, float c2, double *loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NPARAM) {
        double acc = 0.0;
        for (int b = 0; b < nparts; ++b) acc += (double)part[(int64_t)b * NPARAM + p];
        const float g = (float)acc;
        if (grad) grad[p] = g;
        if (m) {
            const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
            const float mp = b1 * m[p] + (1.f - b1) * g;
            const float vp = b2 * v[p] + (1.f - b2) * g * g;
            m[p] = mp;
            v[p] = vp;
            P[p] -= lr * (mp / c1) / (sqrtf(vp / c2) + eps);
        }
    }
    if (p == 0 && loss) {
        double a = 0.0;
        for (int b = 0; b < nparts; ++b) a += loss_part[b];
        *loss = a / (double)n;
    }
}

FeatIn feat_in(const Ctx *c) {
    return FeatIn{c->rp, c->ci, c->diag, c->App, c->ApT, c->ATp, c->lf_base ? c->lf_base : c->St, c->lf_sat};
}

struct TrainBufs {
    float *X = nullptr, *T = nullptr, *part = nullptr;
    double *lpart = nullptr;
    int nparts = 0;
    ~TrainBufs() { dfree(X); dfree(T); dfree(part); dfree(lpart); }
};

cptr_status train_prepare(Ctx *c, const double *feat, const double *target, int32_t n, TrainBufs &B) {
    CPTR_CUDA_TRY(c, cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sizeof(TrainSmem)));
    B.nparts = (int)std::min<int64_t>((n + TS - 1) / TS, kTrainCtas);
    CPTR_TRY(dalloc_t(c, &B.X, (size_t)n * NF));
    CPTR_TRY(dalloc_t(c, &B.T, (size_t)n));
    CPTR_TRY(dalloc_t(c, &B.part, (size_t)B.nparts * NPARAM));
    CPTR_TRY(dalloc_t(c, &B.lpart, (size_t)B.nparts));
    launch_d2f(c, feat, B.X, (int64_t)n * NF);
    launch_d2f(c, target, B.T, n);
    return CPTR_OK;
}

void launch_grad(Ctx *c, const TrainBufs &B, int32_t n, const float *P) {
    (k_mlp_grad<<<B.nparts, TT, sizeof(TrainSmem), c->stream>>>(B.X, B.T, n, P, B.part, B.lpart), note_launch());
}

}  // namespace

cptr_status learned_prepare(Ctx *c) {
    const int32_t n = c->n;
    CPTR_TRY(dalloc_t(c, &c->lf_sat, (size_t)2 * n));
    (k_sat_terms<<<nblk(n, 256), 256, 0, c->stream>>>(n, c->b, c->ps, c->ts, c->diag, c->A, c->lf_sat), note_launch());
    CPTR_CUDA_TRY(c, cudaGetLastError());
    return CPTR_OK;
}

cptr_status learned_schur(Ctx *c, bool *used) {
    *used = false;
    const int32_t n = c->n;
    if (!c->lf_s) CPTR_TRY(dalloc_t(c, &c->lf_s, (size_t)n));
    (k_fill<<<nblk(n, 256), 256, 0, c->stream>>>(c->lf_s, n, 1.0), note_launch());
    if (!c->mlp) return CPTR_OK;
    double *St = nullptr;
    CPTR_TRY(dalloc_t(c, &St, (size_t)c->nnzb));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(c->flag, 0, sizeof(int32_t), c->stream));
    (k_learned_schur<<<nblk(n, 256), 256, 0, c->stream>>>(feat_in(c), n, c->mlp, St, c->lf_s, c->flag), note_launch());
    int32_t bad = 0;
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(&bad, c->flag, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (bad) {
        dfree(St);
        (k_fill<<<nblk(n, 256), 256, 0, c->stream>>>(c->lf_s, n, 1.0), note_launch());
        return CPTR_OK;
    }
    c->lf_base = c->St;   // kept: the features of later calls refer to the base
    c->St = St;
    *used = true;
    return CPTR_OK;
}

cptr_status learned_features(Ctx *c, double *feat) {
    (k_features<<<nblk(c->n, 128), 128, 0, c->stream>>>(feat_in(c), c->n, feat), note_launch());
    CPTR_CUDA_TRY(c, cudaGetLastError());
    return CPTR_OK;
}

cptr_status mlp_infer(Ctx *c, const double *feat, int32_t n, float *y) {
    (k_infer<<<nblk(n, 256), 256, 0, c->stream>>>(feat, n, c->mlp, y), note_launch());
    CPTR_CUDA_TRY(c, cudaGetLastError());
    return CPTR_OK;
}

cptr_status mlp_loss_grad(Ctx *c, const double *feat, const double *target, int32_t n, const float *params,
                          float *grad, double *loss) {
    TrainBufs B;
    CPTR_TRY(train_prepare(c, feat, target, n, B));
    double *dloss = nullptr;
    CPTR_TRY(dalloc_t(c, &dloss, 1));
    launch_grad(c, B, n, params);
    (k_mlp_reduce<<<nblk(NPARAM, 256), 256, 0, c->stream>>>(B.part, B.lpart, B.nparts, n, grad, nullptr, nullptr,
                                                              nullptr, 0.f, 1.f, 1.f, dloss),
     note_launch());
    CPTR_CUDA_TRY(c, cudaGetLastError());
    double l = 0.0;
    cptr_status s = copy_to_host(c, &l, dloss, sizeof(double));
    dfree(dloss);
    if (s != CPTR_OK) return s;
    if (loss) *loss = l;
    return CPTR_OK;
}

cptr_status mlp_train(Ctx *c, const double *feat, const double *target, int32_t n, float *params, int32_t steps,
                      float lr, double *loss_hist) {
    TrainBufs B;
    CPTR_TRY(train_prepare(c, feat, target, n, B));
    float *m = nullptr, *v = nullptr;
    double *dloss = nullptr;
    CPTR_TRY(dalloc_t(c, &m, NPARAM));
    CPTR_TRY(dalloc_t(c, &v, NPARAM));
    CPTR_TRY(dalloc_t(c, &dloss, (size_t)std::max(steps, 1)));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(m, 0, sizeof(float) * NPARAM, c->stream));
    CPTR_CUDA_TRY(c, cudaMemsetAsync(v, 0, sizeof(float) * NPARAM, c->stream));
    for (int32_t k = 1; k <= steps; ++k) {
        const float c1 = (float)(1.0 - pow(0.9, k)), c2 = (float)(1.0 - pow(0.999, k));
        launch_grad(c, B, n, params);
        (k_mlp_reduce<<<nblk(NPARAM, 256), 256, 0, c->stream>>>(B.part, B.lpart, B.nparts, n, nullptr, params, m, v,
                                                                  lr, c1, c2, dloss + (k - 1)),
         note_launch());
    }
    CPTR_CUDA_TRY(c, cudaGetLastError());
    cptr_status s = CPTR_OK;
    if (loss_hist && steps > 0) s = copy_to_host(c, loss_hist, dloss, sizeof(double) * steps);
    else CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    dfree(m);
    dfree(v);
    dfree(dloss);
    return s;
}

}  // namespace cptr
