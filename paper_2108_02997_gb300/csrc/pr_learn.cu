// pr_learn.cu — learned warm start (no counterpart in the paper): per-vertex
// features, a 5-64-64-1 GELU MLP predicting log(N r), its training on the
// device (forward, backward, Adam), and the start vector exp(y)/sum(exp(y)).
//
// The fixed point of the iteration does not depend on the start, so a learned
// start can only change how many updates a solve needs; the uniform start
// remains the default.
//
// Numerics: features FP32; weight matrices held as FP32 master copies and
// BF16 operands; the 64x64 contractions (layer 2 forward, dH1 = dZ2 W2 and
// dW2 = dZ2^T H1) run on tensor cores with warp-level mma.sync m16n8k16
// (BF16 inputs, FP32 accumulation); the 5-wide first layer and the 64-wide
// output layer run on CUDA cores in FP32; biases FP32. Gradients are summed
// per CTA and then over CTAs in a fixed order (deterministic). Training uses
// the exact (erf) GELU; inference, which only has to produce a start vector,
// evaluates GELU by its tanh approximation on the hardware tanh.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <tuple>
#include <vector>

#include "pr_internal.cuh"

namespace {

constexpr int kH = 64;                  // hidden width
constexpr int kF = 5;                   // features per vertex
constexpr int kFS = 8;                  // feature row stride (floats)
constexpr int oW1 = 0, oB1 = oW1 + kH * kF, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH, oB3 = oW3 + kH;
constexpr int kParams = oB3 + 1;        // 4609
constexpr int kMlpThreads = 128;        // 4 warps; each warp owns 16 rows of a 64-row block
constexpr int kRowsPerBlock = 64;
constexpr int kLd = kH + 8;             // padded leading dimension of BF16 tiles (bank spread)

struct MlpDev {
    float *master = nullptr;            // kParams FP32 (the trained values)
    float *m = nullptr, *v = nullptr;   // Adam moments
    __nv_bfloat16 *wbf = nullptr;       // kParams BF16 copies (only W1, W2, W3 are used as BF16)
    float *grad = nullptr;              // kParams + 1 (last: loss)
    float *part = nullptr;              // per-CTA partials, part_ctas x (kParams + 1)
    int part_ctas = 0;
};

}  // namespace

struct pr_mlp {
    uint32_t magic;
    MlpDev d;
    int step;
    // Mean over the training sets of ln(||1/N - r*||_1 / ||r0 - r*||_1): how
    // many e-folds of the start's error the network removes (measured at the
    // end of pr_mlp_train, or set by the caller); PR_INIT_AUTO's input.
    double gain;
    int has_gain;
};

bool pr_mlp_valid(const pr_mlp *m) { return m && registry_has(m) && m->magic == kMlpMagic; }

namespace {

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
// GELU by its tanh approximation (Hendrycks and Gimpel, 2016),
// 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))), with the hardware
// tanh.approx.f32 (one special-function instruction instead of an erf). The
// form is within 4.8e-4 of the exact GELU; with the approximate tanh the
// difference stays far below the BF16 rounding of the hidden activations.
// Used by inference only; training differentiates the exact form.
__device__ __forceinline__ float gelu_tanh(float x) {
    const float u = x * fmaf(0.0356774081f * x, x, 0.7978845608f);
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
    const float hx = 0.5f * x;
    return fmaf(hx, t, hx);
}
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// D = A(16x16, row-major) * B(16x8, given as B^T rows) + D, BF16 in, FP32 accumulate.
// Fragment layout of mma.sync m16n8k16 with g = lane/4, t = lane%4:
//   a0 = A[g][2t..2t+1], a1 = A[g+8][2t..], a2 = A[g][2t+8..], a3 = A[g+8][2t+8..]
//   b0 = B[2t..2t+1][g] = BT[g][2t..],  b1 = BT[g][2t+8..]
//   c0,c1 = D[g][2t], D[g][2t+1];  c2,c3 = D[g+8][2t], D[g+8][2t+1]
__device__ __forceinline__ void mma16816(float *c, const uint32_t *a, const uint32_t *b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }
// A fragment of the 16x16 block at (row0, k0) of a row-major BF16 matrix with leading dim ld.
__device__ __forceinline__ void load_a(uint32_t *a, const __nv_bfloat16 *A, int ld, int row0, int k0, int lane) {
    const int g = lane >> 2, t = lane & 3;
    a[0] = ld32(A + (row0 + g) * ld + k0 + 2 * t);
    a[1] = ld32(A + (row0 + g + 8) * ld + k0 + 2 * t);
    a[2] = ld32(A + (row0 + g) * ld + k0 + 2 * t + 8);
    a[3] = ld32(A + (row0 + g + 8) * ld + k0 + 2 * t + 8);
}
// B fragment of the 16x8 block at (k0, n0) of B, where BT (row-major, N x K) holds B transposed.
__device__ __forceinline__ void load_b(uint32_t *b, const __nv_bfloat16 *BT, int ld, int n0, int k0, int lane) {
    const int g = lane >> 2, t = lane & 3;
    b[0] = ld32(BT + (n0 + g) * ld + k0 + 2 * t);
    b[1] = ld32(BT + (n0 + g) * ld + k0 + 2 * t + 8);
}

struct MlpShared {
    __nv_bfloat16 w2[kH * kLd];         // W2[n][k]
    __nv_bfloat16 w2t[kH * kLd];        // W2^T[n][k] = W2[k][n]
    float w1[kH * kF], b1[kH], b2[kH], w3[kH], b3;
    float f[kRowsPerBlock * kFS];       // features of the block's rows
    float z1[kRowsPerBlock * kH];       // pre-activations of layer 1 (later dZ1)
    __nv_bfloat16 h1[kRowsPerBlock * kLd];    // H1 [row][j]
    __nv_bfloat16 h1t[kH * kLd];              // H1^T [j][row]
    __nv_bfloat16 dz2[kRowsPerBlock * kLd];   // dZ2 [row][i]
    __nv_bfloat16 dz2t[kH * kLd];             // dZ2^T [i][row]
    float y[kRowsPerBlock];
};

__device__ void load_weights(MlpShared &S, const float *master, const __nv_bfloat16 *wbf) {
    for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) {
        const int n = i / kH, k = i % kH;
        const __nv_bfloat16 w = wbf[oW2 + i];
        S.w2[n * kLd + k] = w;
        S.w2t[k * kLd + n] = w;
    }
    for (int i = threadIdx.x; i < kH * kF; i += blockDim.x) S.w1[i] = __bfloat162float(wbf[oW1 + i]);
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        S.b1[i] = master[oB1 + i];
        S.b2[i] = master[oB2 + i];
        S.w3[i] = __bfloat162float(wbf[oW3 + i]);
    }
    if (threadIdx.x == 0) S.b3 = master[oB3];
}

// Forward pass of one 64-row block. Leaves z1 (FP32), h1/h1t (BF16) in shared
// memory, and for each warp the layer-2 accumulators (z2 + b2) in c2, and the
// outputs y in S.y. Rows >= nrows are zero-feature padding.
__device__ void block_forward(MlpShared &S, int nrows, float c2[8][4]) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // layer 1 on CUDA cores: z1[r][j] = b1[j] + sum_f W1[j][f] f[r][f]
    for (int i = tid; i < kRowsPerBlock * kH; i += blockDim.x) {
        const int r = i / kH, j = i % kH;
        float z = S.b1[j];
#pragma unroll
        for (int f = 0; f < kF; f++) z = fmaf(S.w1[j * kF + f], S.f[r * kFS + f], z);
        S.z1[i] = z;
        const __nv_bfloat16 h = __float2bfloat16_rn(gelu(z));
        S.h1[r * kLd + j] = h;
        S.h1t[j * kLd + r] = h;
    }
    __syncthreads();
    // layer 2 on tensor cores: this warp's 16 rows x 64 outputs, K = 64
    const int row0 = warp * 16;
#pragma unroll
    for (int nt = 0; nt < 8; nt++)
#pragma unroll
        for (int q = 0; q < 4; q++) c2[nt][q] = 0.0f;
#pragma unroll
    for (int ks = 0; ks < 4; ks++) {
        uint32_t a[4];
        load_a(a, S.h1, kLd, row0, ks * 16, lane);
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            uint32_t b[2];
            load_b(b, S.w2, kLd, nt * 8, ks * 16, lane);
            mma16816(c2[nt], a, b);
        }
    }
    // z2 + b2, then y = sum_j gelu(z2) w3[j] + b3 (each lane holds rows g and g+8)
    const int g = lane >> 2, t = lane & 3;
    float ylo = 0.0f, yhi = 0.0f;
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
        const int j = nt * 8 + 2 * t;
        c2[nt][0] += S.b2[j];
        c2[nt][1] += S.b2[j + 1];
        c2[nt][2] += S.b2[j];
        c2[nt][3] += S.b2[j + 1];
        ylo = fmaf(gelu(c2[nt][0]), S.w3[j], ylo);
        ylo = fmaf(gelu(c2[nt][1]), S.w3[j + 1], ylo);
        yhi = fmaf(gelu(c2[nt][2]), S.w3[j], yhi);
        yhi = fmaf(gelu(c2[nt][3]), S.w3[j + 1], yhi);
    }
    // the four lanes sharing g hold disjoint columns: add them in a fixed tree
    ylo += __shfl_xor_sync(0xffffffffu, ylo, 1);
    yhi += __shfl_xor_sync(0xffffffffu, yhi, 1);
    ylo += __shfl_xor_sync(0xffffffffu, ylo, 2);
    yhi += __shfl_xor_sync(0xffffffffu, yhi, 2);
    if (t == 0) {
        S.y[row0 + g] = ylo + S.b3;
        S.y[row0 + g + 8] = yhi + S.b3;
    }
    (void)nrows;
}

// ------------------------------------------------------------------ features
// f = [log(1+indeg), log(1+outdeg), mean and max over in-neighbours u of
// log(1+outdeg(u)) (0 without in-neighbours), alpha], relabelled order.
// Rows are relabelled by descending in-degree class, so each of three row
// ranges gets its own worker size: rows with at least kHubDeg in-edges a CTA
// each, rows with at least kWarpDeg a warp each, the rest a thread each.
constexpr int kHubDeg = 2048;
constexpr int kWarpDeg = 32;
constexpr int kFeatThreads = 512;
constexpr int kFeatWarps = kFeatThreads / 32;

// lo[v] = log(1 + outdeg(v)), gathered once per in-edge by the features kernel
__global__ void log_outdeg_kernel(const int32_t *__restrict__ outdeg, int32_t n, float *__restrict__ lo) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
        lo[v] = log1pf((float)outdeg[v]);
}

// One feature row: S = 8 floats (training layout, alpha in f[4], zero pad) or
// S = 4 floats (inference layout, alpha passed to the network kernel).
template <int S>
__device__ __forceinline__ void put_features(float *feat, long long v, int32_t d, float lov, float s, float mx,
                                             float alpha) {
    float *f = feat + (size_t)v * S;
    *reinterpret_cast<float4 *>(f) =
        make_float4(log1pf((float)d), lov, d > 0 ? s / (float)d : 0.0f, d > 0 ? mx : 0.0f);
    if (S == 8) *reinterpret_cast<float4 *>(f + 4) = make_float4(alpha, 0.0f, 0.0f, 0.0f);
}

template <int S>
__global__ void __launch_bounds__(kFeatThreads) features_kernel(const int32_t *__restrict__ off,
                                                                const int32_t *__restrict__ src,
                                                                const float *__restrict__ lo, int32_t n,
                                                                int32_t hub_end, int32_t warp_end, float alpha,
                                                                float *__restrict__ feat) {
    __shared__ float red_s[kFeatWarps], red_m[kFeatWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // rows [0, hub_end): one CTA per row, four independent gathers per thread in flight
    for (int32_t v = blockIdx.x; v < hub_end; v += gridDim.x) {
        const int32_t e0 = off[v], e1 = off[v + 1];
        float s = 0.0f, mx = 0.0f;
        int32_t e = e0 + tid;
        for (; e + 3 * kFeatThreads < e1; e += 4 * kFeatThreads) {
            const int32_t u0 = src[e], u1 = src[e + kFeatThreads], u2 = src[e + 2 * kFeatThreads],
                          u3 = src[e + 3 * kFeatThreads];
            const float x0 = lo[u0], x1 = lo[u1], x2 = lo[u2], x3 = lo[u3];
            s += (x0 + x1) + (x2 + x3);
            mx = fmaxf(mx, fmaxf(fmaxf(x0, x1), fmaxf(x2, x3)));
        }
        for (; e < e1; e += kFeatThreads) {
            const float x = lo[src[e]];
            s += x;
            mx = fmaxf(mx, x);
        }
        for (int m = 16; m > 0; m >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, m);
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, m));
        }
        if (lane == 0) {
            red_s[warp] = s;
            red_m[warp] = mx;
        }
        __syncthreads();
        if (tid == 0) {
            float ts = 0.0f, tm = 0.0f;
            for (int w = 0; w < kFeatWarps; w++) {
                ts += red_s[w];
                tm = fmaxf(tm, red_m[w]);
            }
            put_features<S>(feat, v, e1 - e0, lo[v], ts, tm, alpha);
        }
        __syncthreads();
    }
    // rows [hub_end, warp_end): one warp per row
    const long long nw = (long long)gridDim.x * kFeatWarps;
    for (long long v = hub_end + (long long)blockIdx.x * kFeatWarps + warp; v < warp_end; v += nw) {
        const int32_t e0 = off[v], e1 = off[v + 1];
        float s = 0.0f, mx = 0.0f;
        int32_t e = e0 + lane;
        for (; e + 32 < e1; e += 64) {
            const float x0 = lo[src[e]], x1 = lo[src[e + 32]];
            s += x0 + x1;
            mx = fmaxf(mx, fmaxf(x0, x1));
        }
        if (e < e1) {
            const float x = lo[src[e]];
            s += x;
            mx = fmaxf(mx, x);
        }
        for (int m = 16; m > 0; m >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, m);
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, m));
        }
        if (lane == 0) put_features<S>(feat, v, e1 - e0, lo[v], s, mx, alpha);
    }
    // rows [warp_end, n): one thread per row (fewer than kWarpDeg in-edges each)
    const long long nt = (long long)gridDim.x * kFeatThreads;
    for (long long v = warp_end + (long long)blockIdx.x * kFeatThreads + tid; v < n; v += nt) {
        const int32_t e0 = off[v], e1 = off[v + 1];
        float s = 0.0f, mx = 0.0f;
        int32_t e = e0;
        for (; e + 1 < e1; e += 2) {
            const float x0 = lo[src[e]], x1 = lo[src[e + 1]];
            s += x0 + x1;
            mx = fmaxf(mx, fmaxf(x0, x1));
        }
        if (e < e1) {
            const float x = lo[src[e]];
            s += x;
            mx = fmaxf(mx, x);
        }
        put_features<S>(feat, v, e1 - e0, lo[v], s, mx, alpha);
    }
}

// caller-order copy of the features (n x 5)
__global__ void features_out_kernel(const float *feat, const int32_t *perm, int32_t n, float *out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)n * kF;
         i += (long long)gridDim.x * blockDim.x) {
        const int32_t v = (int32_t)(i / kF), f = (int32_t)(i % kF);
        out[(size_t)perm[v] * kF + f] = feat[(size_t)v * kFS + f];
    }
}

// targets t = log(N r*), relabelled order, from r* in caller order
__global__ void targets_kernel(const double *r_caller, const int32_t *perm, int32_t n, float *t) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
        t[v] = (float)log((double)n * r_caller[perm[v]]);
}

// ------------------------------------------------------------------ inference
// Forward pass without shared-memory activations: each warp takes 16-row
// tiles in turn; a lane computes the layer-1 activations of exactly the
// entries its mma.sync A fragments hold (rows g and g+8, columns 2t, 2t+1,
// 2t+8, 2t+9 of each 16-column block) straight into registers, so only the
// weights sit in shared memory and no CTA-wide barrier separates the layers.
// The arithmetic, and its order, is that of block_forward, with GELU evaluated
// by gelu_tanh. Each CTA also writes the largest y it produced (for the softmax).
constexpr int kInferThreads = 256;
constexpr int kInferWarps = kInferThreads / 32;

struct InferShared {
    __nv_bfloat16 w2[kH * kLd];   // W2[n][k]
    float4 w1[kH];                // W1[j][0..3]
    float w1a[kH];                // W1[j][4] (the alpha weight)
    float b1[kH], b2[kH], w3[kH];
    float b3;
    float wmax[kInferWarps];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

__global__ void __launch_bounds__(kInferThreads, 2) mlp_infer_kernel(const float *master, const __nv_bfloat16 *wbf,
                                                                     const float4 *__restrict__ feat, int32_t n,
                                                                     float alpha, float *__restrict__ y,
                                                                     float *__restrict__ cta_max) {
    __shared__ __align__(16) InferShared S;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < kH * kH; i += kInferThreads) S.w2[(i / kH) * kLd + (i % kH)] = wbf[oW2 + i];
    for (int j = tid; j < kH; j += kInferThreads) {
        const __nv_bfloat16 *w = wbf + oW1 + j * kF;
        S.w1[j] = make_float4(__bfloat162float(w[0]), __bfloat162float(w[1]), __bfloat162float(w[2]),
                              __bfloat162float(w[3]));
        S.w1a[j] = __bfloat162float(w[4]);
        S.b1[j] = master[oB1 + j];
        S.b2[j] = master[oB2 + j];
        S.w3[j] = __bfloat162float(wbf[oW3 + j]);
    }
    if (tid == 0) S.b3 = master[oB3];
    __syncthreads();
    const int g = lane >> 2, t = lane & 3;
    float ymax = -INFINITY;
    const long long ntiles = ((long long)n + 15) / 16;
    for (long long tile = (long long)blockIdx.x * kInferWarps + warp; tile < ntiles;
         tile += (long long)gridDim.x * kInferWarps) {
        const long long ra = tile * 16 + g, rb = ra + 8;
        const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const float4 fa = ra < n ? feat[ra] : zero, fb = rb < n ? feat[rb] : zero;
        float c2[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; nt++)
#pragma unroll
            for (int q = 0; q < 4; q++) c2[nt][q] = 0.0f;
#pragma unroll
        for (int ks = 0; ks < 4; ks++) {
            float ha[4], hb[4];   // columns ks*16 + 2t + {0, 1, 8, 9}
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int j = ks * 16 + 2 * t + (q & 1) + (q >> 1) * 8;
                const float4 w = S.w1[j];
                const float wa = S.w1a[j];
                float za = S.b1[j], zb = za;
                za = fmaf(w.x, fa.x, za);
                zb = fmaf(w.x, fb.x, zb);
                za = fmaf(w.y, fa.y, za);
                zb = fmaf(w.y, fb.y, zb);
                za = fmaf(w.z, fa.z, za);
                zb = fmaf(w.z, fb.z, zb);
                za = fmaf(w.w, fa.w, za);
                zb = fmaf(w.w, fb.w, zb);
                za = fmaf(wa, ra < n ? alpha : 0.0f, za);
                zb = fmaf(wa, rb < n ? alpha : 0.0f, zb);
                ha[q] = gelu_tanh(za);
                hb[q] = gelu_tanh(zb);
            }
            const uint32_t a[4] = {pack_bf16(ha[0], ha[1]), pack_bf16(hb[0], hb[1]), pack_bf16(ha[2], ha[3]),
                                   pack_bf16(hb[2], hb[3])};
#pragma unroll
            for (int nt = 0; nt < 8; nt++) {
                uint32_t b[2];
                load_b(b, S.w2, kLd, nt * 8, ks * 16, lane);
                mma16816(c2[nt], a, b);
            }
        }
        float ylo = 0.0f, yhi = 0.0f;
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            const int j = nt * 8 + 2 * t;
            ylo = fmaf(gelu_tanh(c2[nt][0] + S.b2[j]), S.w3[j], ylo);
            ylo = fmaf(gelu_tanh(c2[nt][1] + S.b2[j + 1]), S.w3[j + 1], ylo);
            yhi = fmaf(gelu_tanh(c2[nt][2] + S.b2[j]), S.w3[j], yhi);
            yhi = fmaf(gelu_tanh(c2[nt][3] + S.b2[j + 1]), S.w3[j + 1], yhi);
        }
        ylo += __shfl_xor_sync(0xffffffffu, ylo, 1);
        yhi += __shfl_xor_sync(0xffffffffu, yhi, 1);
        ylo += __shfl_xor_sync(0xffffffffu, ylo, 2);
        yhi += __shfl_xor_sync(0xffffffffu, yhi, 2);
        ylo += S.b3;
        yhi += S.b3;
        if (t == 0) {
            if (ra < n) {
                y[ra] = ylo;
                ymax = fmaxf(ymax, ylo);
            }
            if (rb < n) {
                y[rb] = yhi;
                ymax = fmaxf(ymax, yhi);
            }
        }
    }
    for (int m = 16; m > 0; m >>= 1) ymax = fmaxf(ymax, __shfl_xor_sync(0xffffffffu, ymax, m));
    if (lane == 0) S.wmax[warp] = ymax;
    __syncthreads();
    if (tid == 0) {
        float m = -INFINITY;
        for (int w = 0; w < kInferWarps; w++) m = fmaxf(m, S.wmax[w]);
        cta_max[blockIdx.x] = m;
    }
}

// exp(y - max) summed in FP64 per CTA, then r0 = exp(y - max) / sum
__global__ void expsum_kernel(const float *y, int32_t n, const float *block_max, int nblocks, double *block_sum) {
    __shared__ double s[256];
    __shared__ float gmax;
    if (threadIdx.x == 0) {
        float m = -INFINITY;
        for (int b = 0; b < nblocks; b++) m = fmaxf(m, block_max[b]);
        gmax = m;
    }
    __syncthreads();
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += (double)expf(y[i] - gmax);
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) block_sum[blockIdx.x] = s[0];
}
// perm == nullptr: r0 in relabelled order; else r0[perm[v]] (caller order)
__global__ void normalise_kernel(const float *y, int32_t n, const float *block_max, int nmax, const double *block_sum,
                                 int nsum, const int32_t *perm, double *r0) {
    __shared__ float gmax;
    __shared__ double total;
    if (threadIdx.x == 0) {
        float m = -INFINITY;
        for (int b = 0; b < nmax; b++) m = fmaxf(m, block_max[b]);
        double t = 0.0;
        for (int b = 0; b < nsum; b++) t += block_sum[b];
        gmax = m;
        total = t;
    }
    __syncthreads();
    const bool ok = total > 0.0 && isfinite(total) && isfinite(gmax);
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        const double x = ok ? (double)expf(y[v] - gmax) / total : 1.0 / (double)n;
        r0[perm ? perm[v] : v] = x;
    }
}

// ------------------------------------------------------------------ training
// Forward + backward of mean((y - t)^2) over all n rows; per-CTA partial
// gradients (kParams floats) and loss, in part[cta][...].
__global__ void __launch_bounds__(kMlpThreads) mlp_grad_kernel(const float *master, const __nv_bfloat16 *wbf,
                                                               const float *feat, const float *target, int32_t n,
                                                               float *part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpShared &S = *reinterpret_cast<MlpShared *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int row0 = warp * 16;
    load_weights(S, master, wbf);
    const float inv_n = 1.0f / (float)n;
    // per-thread accumulators
    float acc_w2[8][4];                 // dW2 rows [16 warp .. +16) x 64 cols (mma layout)
#pragma unroll
    for (int nt = 0; nt < 8; nt++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc_w2[nt][q] = 0.0f;
    float acc_b2[16], acc_w3[16];       // columns nt*8 + 2t + {0,1}
#pragma unroll
    for (int q = 0; q < 16; q++) acc_b2[q] = acc_w3[q] = 0.0f;
    float acc_b3 = 0.0f, acc_loss = 0.0f;
    // dW1 / db1: thread j = tid % 64 owns column j; threads tid < 64 rows 0..31, others 32..63
    float acc_w1[kF], acc_b1 = 0.0f;
#pragma unroll
    for (int f = 0; f < kF; f++) acc_w1[f] = 0.0f;

    for (long long b0 = (long long)blockIdx.x * kRowsPerBlock; b0 < n; b0 += (long long)gridDim.x * kRowsPerBlock) {
        const int nrows = (int)min((long long)kRowsPerBlock, (long long)n - b0);
        __syncthreads();
        for (int i = tid; i < kRowsPerBlock * kFS; i += blockDim.x) {
            const int r = i / kFS;
            S.f[i] = r < nrows ? feat[(size_t)(b0 + r) * kFS + (i % kFS)] : 0.0f;
        }
        __syncthreads();
        float c2[8][4];
        block_forward(S, nrows, c2);
        __syncthreads();
        // dy = 2 (y - t) / n for valid rows (padding rows contribute nothing)
        const int rlo = row0 + g, rhi = row0 + g + 8;
        float dylo = 0.0f, dyhi = 0.0f;
        if (rlo < nrows) {
            const float e = S.y[rlo] - target[b0 + rlo];
            dylo = 2.0f * e * inv_n;
            if (t == 0) acc_loss = fmaf(e * e, inv_n, acc_loss);
        }
        if (rhi < nrows) {
            const float e = S.y[rhi] - target[b0 + rhi];
            dyhi = 2.0f * e * inv_n;
            if (t == 0) acc_loss = fmaf(e * e, inv_n, acc_loss);
        }
        if (t == 0) acc_b3 += dylo + dyhi;
        // output layer and dZ2 = dy * w3 * gelu'(z2)
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const int j = nt * 8 + 2 * t + q;
                acc_w3[nt * 2 + q] = fmaf(dylo, gelu(c2[nt][q]), acc_w3[nt * 2 + q]);
                acc_w3[nt * 2 + q] = fmaf(dyhi, gelu(c2[nt][2 + q]), acc_w3[nt * 2 + q]);
                const float dlo = dylo * S.w3[j] * gelu_grad(c2[nt][q]);
                const float dhi = dyhi * S.w3[j] * gelu_grad(c2[nt][2 + q]);
                acc_b2[nt * 2 + q] += dlo + dhi;
                const __nv_bfloat16 blo = __float2bfloat16_rn(dlo), bhi = __float2bfloat16_rn(dhi);
                S.dz2[rlo * kLd + j] = blo;
                S.dz2[rhi * kLd + j] = bhi;
                S.dz2t[j * kLd + rlo] = blo;
                S.dz2t[j * kLd + rhi] = bhi;
            }
        }
        __syncthreads();
        // dH1 = dZ2 W2 for this warp's rows (tensor cores), dZ1 = dH1 * gelu'(z1) -> S.z1
        {
            float c[8][4];
#pragma unroll
            for (int nt = 0; nt < 8; nt++)
#pragma unroll
                for (int q = 0; q < 4; q++) c[nt][q] = 0.0f;
#pragma unroll
            for (int ks = 0; ks < 4; ks++) {
                uint32_t a[4];
                load_a(a, S.dz2, kLd, row0, ks * 16, lane);
#pragma unroll
                for (int nt = 0; nt < 8; nt++) {
                    uint32_t b[2];
                    load_b(b, S.w2t, kLd, nt * 8, ks * 16, lane);   // B[k=i][n=j] = W2[i][j]
                    mma16816(c[nt], a, b);
                }
            }
#pragma unroll
            for (int nt = 0; nt < 8; nt++)
#pragma unroll
                for (int q = 0; q < 2; q++) {
                    const int j = nt * 8 + 2 * t + q;
                    float &zlo = S.z1[rlo * kH + j];
                    float &zhi = S.z1[rhi * kH + j];
                    zlo = rlo < nrows ? c[nt][q] * gelu_grad(zlo) : 0.0f;
                    zhi = rhi < nrows ? c[nt][2 + q] * gelu_grad(zhi) : 0.0f;
                }
        }
        // dW2[i][j] += sum_r dZ2[r][i] H1[r][j]: warp owns i in [16w, 16w+16), K = 64 rows
#pragma unroll
        for (int ks = 0; ks < 4; ks++) {
            uint32_t a[4];
            load_a(a, S.dz2t, kLd, row0, ks * 16, lane);            // A[i][r] = dZ2^T
#pragma unroll
            for (int nt = 0; nt < 8; nt++) {
                uint32_t b[2];
                load_b(b, S.h1t, kLd, nt * 8, ks * 16, lane);        // B[k=r][n=j] = H1[r][j]
                mma16816(acc_w2[nt], a, b);
            }
        }
        __syncthreads();
        // dW1 / db1 on CUDA cores from dZ1 (S.z1) and the features
        {
            const int j = tid % kH, rbeg = (tid / kH) * (kRowsPerBlock / 2);
            for (int r = rbeg; r < rbeg + kRowsPerBlock / 2; r++) {
                const float d = S.z1[r * kH + j];
                acc_b1 += d;
#pragma unroll
                for (int f = 0; f < kF; f++) acc_w1[f] = fmaf(d, S.f[r * kFS + f], acc_w1[f]);
            }
        }
    }
    __syncthreads();
    // ---- per-CTA partials, written in a fixed layout
    float *P = part + (size_t)blockIdx.x * (kParams + 1);
    // dW2: warp w rows [16w, 16w+16)
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
        const int j = nt * 8 + 2 * t;
        P[oW2 + (row0 + g) * kH + j] = acc_w2[nt][0];
        P[oW2 + (row0 + g) * kH + j + 1] = acc_w2[nt][1];
        P[oW2 + (row0 + g + 8) * kH + j] = acc_w2[nt][2];
        P[oW2 + (row0 + g + 8) * kH + j + 1] = acc_w2[nt][3];
    }
    // b2 / w3 columns: reduce over g (lanes with equal t), then over warps via shared memory
    float *red = S.z1;   // reuse: [4 warps][2 * 64]
#pragma unroll
    for (int q = 0; q < 16; q++) {
        float vb = acc_b2[q], vw = acc_w3[q];
        for (int m = 4; m < 32; m <<= 1) {
            vb += __shfl_xor_sync(0xffffffffu, vb, m);
            vw += __shfl_xor_sync(0xffffffffu, vw, m);
        }
        if (g == 0) {
            const int j = (q / 2) * 8 + 2 * t + (q % 2);
            red[warp * 2 * kH + j] = vb;
            red[warp * 2 * kH + kH + j] = vw;
        }
    }
    // b3 and loss: lanes with t == 0 hold them
    float vb3 = acc_b3, vl = acc_loss;
    for (int m = 1; m < 32; m <<= 1) {
        vb3 += __shfl_xor_sync(0xffffffffu, vb3, m);
        vl += __shfl_xor_sync(0xffffffffu, vl, m);
    }
    __shared__ float s_b3[4], s_loss[4];
    if (lane == 0) {
        s_b3[warp] = vb3;
        s_loss[warp] = vl;
    }
    // dW1/db1: two threads per column, rows halves
    __shared__ float s_w1[2][kH * kF + kH];
    {
        const int j = tid % kH, h = tid / kH;
#pragma unroll
        for (int f = 0; f < kF; f++) s_w1[h][j * kF + f] = acc_w1[f];
        s_w1[h][kH * kF + j] = acc_b1;
    }
    __syncthreads();
    for (int i = tid; i < kH; i += blockDim.x) {
        float vb = 0.0f, vw = 0.0f;
        for (int w = 0; w < 4; w++) {
            vb += red[w * 2 * kH + i];
            vw += red[w * 2 * kH + kH + i];
        }
        P[oB2 + i] = vb;
        P[oW3 + i] = vw;
    }
    for (int i = tid; i < kH * kF; i += blockDim.x) P[oW1 + i] = s_w1[0][i] + s_w1[1][i];
    for (int i = tid; i < kH; i += blockDim.x) P[oB1 + i] = s_w1[0][kH * kF + i] + s_w1[1][kH * kF + i];
    if (tid == 0) {
        P[oB3] = s_b3[0] + s_b3[1] + s_b3[2] + s_b3[3];
        P[kParams] = s_loss[0] + s_loss[1] + s_loss[2] + s_loss[3];
    }
}

// grad[i] = sum over CTAs of part[c][i] (fixed order)
__global__ void reduce_parts_kernel(const float *part, int nparts, float *grad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= kParams; i += gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int c = 0; c < nparts; c++) s += part[(size_t)c * (kParams + 1) + i];
        grad[i] = s;
    }
}

// Adam (Kingma and Ba, 2015) on the FP32 master weights, then BF16 copies.
__global__ void adam_kernel(float *master, float *m, float *v, __nv_bfloat16 *wbf, const float *grad, float lr,
                            float bc1, float bc2) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kParams; i += gridDim.x * blockDim.x) {
        const float gi = grad[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float p = master[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        master[i] = p;
        wbf[i] = __float2bfloat16_rn(p);
    }
}

__global__ void to_bf16_kernel(const float *master, __nv_bfloat16 *wbf) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kParams; i += gridDim.x * blockDim.x)
        wbf[i] = __float2bfloat16_rn(master[i]);
}

// ------------------------------------------------------------------ host helpers
using DBuf = PoolBuf;

pr_status dmalloc(DBuf &b, size_t bytes, cudaStream_t st) { return b.alloc(bytes ? bytes : 16, st); }

int grid_for(long long work, int threads) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long want = (work + threads - 1) / threads;
    return (int)std::max<long long>(1, std::min<long long>(want, (long long)sms * 8));
}

// The training kernel's dynamic shared-memory opt-in, once per device (an
// attribute of the device context).
pr_status mlp_setup_smem() {
    static std::mutex mu;
    static std::set<int> done;
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (!done.count(dev)) {
        PR_CUDA(cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MlpShared)));
        done.insert(dev);
    }
    return PR_OK;
}

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// Features of g at alpha into feat (relabelled order, S floats per row; see
// put_features). The row ranges of the three worker sizes follow from the
// in-degree classes, which are in descending order.
template <int S>
pr_status compute_features_t(const pr_graph *g, double alpha, float *feat, cudaStream_t st) {
    const int32_t n = g->n;
    int32_t hub_end = n, warp_end = n;
    for (const ClassRange &c : g->classes) {
        if (c.max_deg < kHubDeg && hub_end == n) hub_end = c.begin;
        if (c.max_deg < kWarpDeg && warp_end == n) warp_end = c.begin;
    }
    if (hub_end > warp_end) hub_end = warp_end;
    DBuf lo;
    pr_status s = dmalloc(lo, (size_t)n * sizeof(float), st);
    if (s != PR_OK) return s;
    log_outdeg_kernel<<<grid_for(n, 256), 256, 0, st>>>(g->d_outdeg, n, (float *)lo.p);
    PR_CUDA(cudaGetLastError());
    const int blocks = std::max(1, sm_count() * (2048 / kFeatThreads));
    features_kernel<S><<<blocks, kFeatThreads, 0, st>>>(g->d_off, g->d_src, (const float *)lo.p, n, hub_end, warp_end,
                                                        (float)alpha, feat);
    PR_CUDA(cudaGetLastError());
    return PR_OK;
}

// training layout: n x kFS floats
pr_status compute_features(const pr_graph *g, double alpha, float *feat, cudaStream_t st) {
    return compute_features_t<kFS>(g, alpha, feat, st);
}

int mlp_grid(int32_t n) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long blocks = ((long long)n + kRowsPerBlock - 1) / kRowsPerBlock;
    return (int)std::max<long long>(1, std::min<long long>(blocks, (long long)sms * 2));
}

pr_status ensure_parts(pr_mlp *m, int ctas) {
    if (m->d.part_ctas >= ctas) return PR_OK;
    if (m->d.part) cudaFree(m->d.part);
    m->d.part = nullptr;
    m->d.part_ctas = 0;
    PR_CUDA(cudaMalloc((void **)&m->d.part, (size_t)ctas * (kParams + 1) * sizeof(float)));
    m->d.part_ctas = ctas;
    return PR_OK;
}

// full-batch loss and gradient over one (graph, features, targets) set into m->d.grad
pr_status loss_grad(pr_mlp *m, const float *feat, const float *target, int32_t n, cudaStream_t st) {
    pr_status s = mlp_setup_smem();
    if (s != PR_OK) return s;
    const int ctas = mlp_grid(n);
    if ((s = ensure_parts(m, ctas)) != PR_OK) return s;
    mlp_grad_kernel<<<ctas, kMlpThreads, sizeof(MlpShared), st>>>(m->d.master, m->d.wbf, feat, target, n, m->d.part);
    PR_CUDA(cudaGetLastError());
    reduce_parts_kernel<<<(kParams + 256) / 256, 256, 0, st>>>(m->d.part, ctas, m->d.grad);
    PR_CUDA(cudaGetLastError());
    return PR_OK;
}

// Per-CTA partial sums of |r0[v] - t[v]| and |1/n - t[v]| (FP64, fixed
// order within a CTA); r0 and t both in caller order.
__global__ void start_error_kernel(const double *__restrict__ r0, const double *__restrict__ t, int32_t n,
                                   double *__restrict__ part) {
    __shared__ double s_a[256], s_b[256];
    double a = 0.0, b = 0.0;
    const double u = 1.0 / (double)n;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        a += fabs(r0[v] - t[v]);
        b += fabs(u - t[v]);
    }
    s_a[threadIdx.x] = a;
    s_b[threadIdx.x] = b;
    __syncthreads();
    for (int m = 128; m > 0; m >>= 1) {
        if ((int)threadIdx.x < m) {
            s_a[threadIdx.x] += s_a[threadIdx.x + m];
            s_b[threadIdx.x] += s_b[threadIdx.x + m];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s_a[0];
        part[2 * blockIdx.x + 1] = s_b[0];
    }
}

// ln(e_uniform / e_learned) of one (graph, alpha, target) set.
pr_status start_gain(const pr_mlp *m, const pr_graph *g, double alpha, const double *target, cudaStream_t st,
                     double *out) {
    const int32_t n = g->n;
    DBuf r0, part;
    const int ctas = std::max(1, std::min(grid_for(n, 256), 1024));
    pr_status s = dmalloc(r0, (size_t)n * sizeof(double), st);
    if (s == PR_OK) s = dmalloc(part, 2 * (size_t)ctas * sizeof(double), st);
    if (s == PR_OK) s = pr_learned_start(m, g, alpha, (double *)r0.p, false, st);
    if (s != PR_OK) return s;
    start_error_kernel<<<ctas, 256, 0, st>>>((const double *)r0.p, target, n, (double *)part.p);
    PR_CUDA(cudaGetLastError());
    std::vector<double> h(2 * (size_t)ctas);
    PR_CUDA(cudaMemcpyAsync(h.data(), part.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    PR_CUDA(cudaStreamSynchronize(st));
    double el = 0.0, eu = 0.0;
    for (int c = 0; c < ctas; c++) {
        el += h[2 * c];
        eu += h[2 * c + 1];
    }
    *out = (el > 0.0 && eu > 0.0) ? std::log(eu / el) : 0.0;
    return PR_OK;
}

void free_mlp(pr_mlp *m) {
    if (!m) return;
    cudaFree(m->d.master);
    cudaFree(m->d.m);
    cudaFree(m->d.v);
    cudaFree(m->d.wbf);
    cudaFree(m->d.grad);
    cudaFree(m->d.part);
    m->magic = 0;
    delete m;
}

}  // namespace

size_t pr_learned_features_bytes(const pr_graph *g) { return (size_t)g->n * 4 * sizeof(float); }

// inference layout: n rows of 4 floats (alpha passed to the network kernel)
pr_status pr_learned_features(const pr_graph *g, void *feat, cudaStream_t st) {
    return compute_features_t<4>(g, 0.0, static_cast<float *>(feat), st);
}

// Start vector for (g, alpha): features -> MLP -> exp(y - max) / sum.
// Stream-ordered: the caller synchronises when it needs the values on the host.
pr_status pr_learned_start(const pr_mlp *m, const pr_graph *g, double alpha, double *d_out, bool relabelled,
                           cudaStream_t st, const void *feat_in) {
    if (!pr_mlp_valid(m)) return pr_fail(PR_ESTATE, "not a live pr_mlp handle");
    if (!pr_graph_valid(g)) return pr_fail(PR_ESTATE, "not a live graph handle");
    const int32_t n = g->n;
    DBuf feat, y, bmax, bsum;
    pr_status s;
    if (!feat_in) {
        if ((s = dmalloc(feat, pr_learned_features_bytes(g), st)) != PR_OK) return s;
        if ((s = pr_learned_features(g, feat.p, st)) != PR_OK) return s;
        feat_in = feat.p;
    }
    const long long ntiles = ((long long)n + 15) / 16;
    const int ictas = (int)std::max<long long>(
        1, std::min<long long>((ntiles + kInferWarps - 1) / kInferWarps, (long long)sm_count() * 2));
    const int rb = grid_for(n, 256);
    if ((s = dmalloc(y, (size_t)n * sizeof(float), st)) != PR_OK) return s;
    if ((s = dmalloc(bmax, ictas * sizeof(float), st)) != PR_OK) return s;
    if ((s = dmalloc(bsum, rb * sizeof(double), st)) != PR_OK) return s;
    mlp_infer_kernel<<<ictas, kInferThreads, 0, st>>>(m->d.master, m->d.wbf, (const float4 *)feat_in, n, (float)alpha,
                                                      (float *)y.p, (float *)bmax.p);
    PR_CUDA(cudaGetLastError());
    expsum_kernel<<<rb, 256, 0, st>>>((const float *)y.p, n, (const float *)bmax.p, ictas, (double *)bsum.p);
    normalise_kernel<<<rb, 256, 0, st>>>((const float *)y.p, n, (const float *)bmax.p, ictas, (const double *)bsum.p,
                                         rb, relabelled ? nullptr : g->d_perm, d_out);
    PR_CUDA(cudaGetLastError());
    return PR_OK;
}

extern "C" pr_status pr_mlp_create(const float *params, pr_mlp **out) {
    pr_clear_error();
    if (!out) return pr_fail(PR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params) return pr_fail(PR_EINVAL, "params is NULL");
    for (int i = 0; i < kParams; i++)
        if (!std::isfinite(params[i])) return pr_fail(PR_EINVAL, "params must be finite");
    pr_mlp *m = new (std::nothrow) pr_mlp();
    if (!m) return pr_fail(PR_ENOMEM, "host allocation failed");
    m->magic = kMlpMagic;
    m->step = 0;
    m->gain = 0.0;
    m->has_gain = 0;
    cudaError_t e = cudaMalloc((void **)&m->d.master, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->d.m, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->d.v, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->d.wbf, kParams * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->d.grad, (kParams + 1) * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(m->d.master, params, kParams * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->d.m, 0, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(m->d.v, 0, kParams * sizeof(float));
    if (e == cudaSuccess) {
        to_bf16_kernel<<<(kParams + 255) / 256, 256>>>(m->d.master, m->d.wbf);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_mlp(m);
        return pr_cuda_fail(e, "pr_mlp_create");
    }
    registry_add(m);
    *out = m;
    return PR_OK;
}

extern "C" pr_status pr_mlp_destroy(pr_mlp *m) {
    pr_clear_error();
    if (!m) return PR_OK;
    if (!pr_mlp_valid(m)) return pr_fail(PR_ESTATE, "not a live pr_mlp handle");
    registry_remove(m);
    free_mlp(m);
    return PR_OK;
}

extern "C" pr_status pr_mlp_get_params(const pr_mlp *m, float *params_out) {
    pr_clear_error();
    if (!pr_mlp_valid(m)) return pr_fail(PR_ESTATE, "not a live pr_mlp handle");
    if (!params_out) return pr_fail(PR_EINVAL, "params_out is NULL");
    PR_CUDA(cudaMemcpy(params_out, m->d.master, kParams * sizeof(float), cudaMemcpyDeviceToHost));
    return PR_OK;
}

extern "C" pr_status pr_features(const pr_graph *g, double alpha, float *d_feat_out, void *stream) {
    pr_clear_error();
    if (!pr_graph_valid(g)) return pr_fail(PR_ESTATE, "not a live graph handle");
    if (!d_feat_out) return pr_fail(PR_EINVAL, "d_feat_out is NULL");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    DBuf feat;
    pr_status s = dmalloc(feat, (size_t)g->n * kFS * sizeof(float), st);
    if (s != PR_OK) return s;
    if ((s = compute_features(g, alpha, (float *)feat.p, st)) != PR_OK) return s;
    features_out_kernel<<<grid_for((long long)g->n * kF, 256), 256, 0, st>>>((const float *)feat.p, g->d_perm, g->n, d_feat_out);
    PR_CUDA(cudaGetLastError());
    PR_CUDA(cudaStreamSynchronize(st));
    return PR_OK;
}

extern "C" pr_status pr_mlp_warm_start(const pr_mlp *m, const pr_graph *g, double alpha, double *d_r0_out, void *stream) {
    pr_clear_error();
    if (!d_r0_out) return pr_fail(PR_EINVAL, "d_r0_out is NULL");
    if (!(alpha >= 0.0 && alpha <= 1.0)) return pr_fail(PR_EINVAL, "alpha must be in [0, 1]");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    pr_status s = pr_learned_start(m, g, alpha, d_r0_out, false, st);
    if (s != PR_OK) return s;
    PR_CUDA(cudaStreamSynchronize(st));
    return PR_OK;
}

extern "C" pr_status pr_mlp_loss_grad(const pr_mlp *m, const pr_graph *g, double alpha, const double *d_target_r,
                                      float *loss_out, float *grad_out, void *stream) {
    pr_clear_error();
    if (!pr_mlp_valid(m)) return pr_fail(PR_ESTATE, "not a live pr_mlp handle");
    if (!pr_graph_valid(g)) return pr_fail(PR_ESTATE, "not a live graph handle");
    if (!d_target_r) return pr_fail(PR_EINVAL, "d_target_r is NULL");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int32_t n = g->n;
    DBuf feat, tgt;
    pr_status s = dmalloc(feat, (size_t)n * kFS * sizeof(float), st);
    if (s != PR_OK) return s;
    if ((s = dmalloc(tgt, (size_t)n * sizeof(float), st)) != PR_OK) return s;
    if ((s = compute_features(g, alpha, (float *)feat.p, st)) != PR_OK) return s;
    targets_kernel<<<grid_for(n, 256), 256, 0, st>>>(d_target_r, g->d_perm, n, (float *)tgt.p);
    PR_CUDA(cudaGetLastError());
    pr_mlp *mm = const_cast<pr_mlp *>(m);
    if ((s = loss_grad(mm, (const float *)feat.p, (const float *)tgt.p, n, st)) != PR_OK) return s;
    std::vector<float> host(kParams + 1);
    PR_CUDA(cudaMemcpyAsync(host.data(), m->d.grad, (kParams + 1) * sizeof(float), cudaMemcpyDeviceToHost, st));
    PR_CUDA(cudaStreamSynchronize(st));
    if (grad_out) std::memcpy(grad_out, host.data(), kParams * sizeof(float));
    if (loss_out) *loss_out = host[kParams];
    return PR_OK;
}

extern "C" pr_status pr_mlp_train(pr_mlp *m, const pr_graph *const *graphs, const double *alphas,
                                  const double *const *targets, int32_t nsets, int32_t epochs, float lr,
                                  float *loss_out, void *stream) {
    pr_clear_error();
    if (!pr_mlp_valid(m)) return pr_fail(PR_ESTATE, "not a live pr_mlp handle");
    if (nsets < 1 || !graphs || !alphas || !targets) return pr_fail(PR_EINVAL, "need at least one (graph, alpha, target) set");
    if (epochs < 0) return pr_fail(PR_EINVAL, "epochs must be >= 0");
    if (!(lr > 0.0f) || !std::isfinite(lr)) return pr_fail(PR_EINVAL, "lr must be positive and finite");
    for (int i = 0; i < nsets; i++) {
        if (!pr_graph_valid(graphs[i])) return pr_fail(PR_ESTATE, "not a live graph handle in graphs[]");
        if (!targets[i]) return pr_fail(PR_EINVAL, "targets[] entry is NULL");
        if (!(alphas[i] >= 0.0 && alphas[i] <= 1.0)) return pr_fail(PR_EINVAL, "alpha must be in [0, 1]");
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    std::vector<DBuf> feats(nsets), tgts(nsets);
    pr_status s;
    for (int i = 0; i < nsets; i++) {
        const int32_t n = graphs[i]->n;
        if ((s = dmalloc(feats[i], (size_t)n * kFS * sizeof(float), st)) != PR_OK) return s;
        if ((s = dmalloc(tgts[i], (size_t)n * sizeof(float), st)) != PR_OK) return s;
        if ((s = compute_features(graphs[i], alphas[i], (float *)feats[i].p, st)) != PR_OK) return s;
        targets_kernel<<<grid_for(n, 256), 256, 0, st>>>(targets[i], graphs[i]->d_perm, n, (float *)tgts[i].p);
        PR_CUDA(cudaGetLastError());
    }
    std::vector<float> last_loss(nsets, 0.0f);
    for (int ep = 0; ep < epochs; ep++) {
        for (int i = 0; i < nsets; i++) {
            if ((s = loss_grad(m, (const float *)feats[i].p, (const float *)tgts[i].p, graphs[i]->n, st)) != PR_OK) return s;
            m->step++;
            const float bc1 = 1.0f - powf(0.9f, (float)m->step), bc2 = 1.0f - powf(0.999f, (float)m->step);
            adam_kernel<<<(kParams + 255) / 256, 256, 0, st>>>(m->d.master, m->d.m, m->d.v, m->d.wbf, m->d.grad, lr, bc1, bc2);
            PR_CUDA(cudaGetLastError());
            if (ep == epochs - 1)
                PR_CUDA(cudaMemcpyAsync(&last_loss[i], m->d.grad + kParams, sizeof(float), cudaMemcpyDeviceToHost, st));
        }
    }
    PR_CUDA(cudaStreamSynchronize(st));
    if (loss_out) {
        float t = 0.0f;
        for (float x : last_loss) t += x;
        *loss_out = t / (float)nsets;
    }
    // the trained network's gain over the uniform start on its own sets
    if (epochs > 0) {
        double sum = 0.0;
        for (int i = 0; i < nsets; i++) {
            double gi = 0.0;
            if ((s = start_gain(m, graphs[i], alphas[i], targets[i], st, &gi)) != PR_OK) return s;
            sum += gi;
        }
        m->gain = sum / (double)nsets;
        m->has_gain = 1;
    }
    return PR_OK;
}

extern "C" pr_status pr_mlp_gain(const pr_mlp *m, double *gain_out, int32_t *known_out) {
    pr_clear_error();
    if (!pr_mlp_valid(m)) return pr_fail(PR_ESTATE, "not a live pr_mlp handle");
    if (gain_out) *gain_out = m->gain;
    if (known_out) *known_out = m->has_gain;
    return PR_OK;
}

extern "C" pr_status pr_mlp_set_gain(pr_mlp *m, double gain) {
    pr_clear_error();
    if (!pr_mlp_valid(m)) return pr_fail(PR_ESTATE, "not a live pr_mlp handle");
    if (!std::isfinite(gain)) return pr_fail(PR_EINVAL, "gain must be finite");
    m->gain = gain;
    m->has_gain = 1;
    return PR_OK;
}

double pr_mlp_gain_value(const pr_mlp *m) { return m && m->has_gain ? m->gain : 0.0; }

// Device time of the learned start on g (CUDA events): the features, once per
// graph, and the network with its softmax, once per alpha. Measured on the
// first request per device and graph signature and kept.
pr_status pr_learned_cost(const pr_mlp *m, const pr_graph *g, cudaStream_t st, double *feat_us, double *net_us) {
    static std::mutex mu;
    static std::map<std::tuple<int, uint64_t, int32_t>, std::pair<double, double>> cache;
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    const auto key = std::make_tuple(dev, g->signature, g->n);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            *feat_us = it->second.first;
            *net_us = it->second.second;
            return PR_OK;
        }
    }
    DBuf feat, r0;
    pr_status s = dmalloc(feat, pr_learned_features_bytes(g), st);
    if (s == PR_OK) s = dmalloc(r0, (size_t)g->n * sizeof(double), st);
    if (s != PR_OK) return s;
    cudaEvent_t e0, e1, e2;
    PR_CUDA(cudaEventCreate(&e0));
    PR_CUDA(cudaEventCreate(&e1));
    PR_CUDA(cudaEventCreate(&e2));
    struct EvG { cudaEvent_t a, b, c; ~EvG() { cudaEventDestroy(a); cudaEventDestroy(b); cudaEventDestroy(c); } } evg{e0, e1, e2};
    // one untimed round (first launches), then the timed one
    for (int round = 0; round < 2; round++) {
        PR_CUDA(cudaEventRecord(e0, st));
        if ((s = pr_learned_features(g, feat.p, st)) != PR_OK) return s;
        PR_CUDA(cudaEventRecord(e1, st));
        if ((s = pr_learned_start(m, g, 0.85, (double *)r0.p, true, st, feat.p)) != PR_OK) return s;
        PR_CUDA(cudaEventRecord(e2, st));
    }
    PR_CUDA(cudaEventSynchronize(e2));
    float f = 0.f, t = 0.f;
    PR_CUDA(cudaEventElapsedTime(&f, e0, e1));
    PR_CUDA(cudaEventElapsedTime(&t, e1, e2));
    *feat_us = 1e3 * f;
    *net_us = 1e3 * t;
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = {*feat_us, *net_us};
    return PR_OK;
}
