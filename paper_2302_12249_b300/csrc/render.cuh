// render.cuh -- fused per-ray render kernel and traversal-only kernel for sm_103a.
//
// One thread renders one pixel ray end to end: ray generation, segment table, lattice walk
// with a per-sample finest-cell test and coarse-to-fine empty-space skipping, gather of the 20
// texels of each evaluated sample, all eight channels interpolated in one tap-major pass (the
// appearance values enter the result only when the sample's opacity is non-zero, Sec. 5),
// front-to-back compositing of C_d and F with early termination (Eq. 1, Eq. 2, Sec. 5), and
// finally the deferred MLP h(C_d, F, d) (Sec. 2, App. B), whose 883 weights reach each CTA's
// shared memory by one bulk (TMA) copy that overlaps the march (FP32: per pixel on the CUDA
// cores; FP16 / BF16: the CTA's 128 pixels as one M = 128 tcgen05.mma tile, accumulated in
// tensor memory).  A warp covers an 8 x 4 pixel tile and a CTA a 16 x 8 tile, so neighbouring
// rays walk neighbouring texels together and share L1 lines.  Template parameters select the storage
// (uint8 block-sparse / dense float), the precision (FP32 / FP16 / BF16 appearance arithmetic
// and MLP), the gather geometry (the paper's / grid-only / run-time strides) and the contraction
// (contract_pi, or the spherical ablation's dense march).
#pragma once

#include "field.cuh"
#include "traverse.cuh"
#include "umma.cuh"

namespace merf {

constexpr int kMaxCams = 32;        // cameras per launch (passed by value)
constexpr int kMlpParams = 883;
constexpr int kTileW = 16, kTileH = 8, kThreads = 128;
constexpr int kAuxSize = 12;

struct CamBlock {
    float m[kMaxCams][16];
};

struct RenderParams {
    FieldView fv;
    OccView occ;
    const float *mlp;
    float *out;                       // [n][H][W][3]
    float *aux;                       // [n][H][W][kAuxSize] or null
    unsigned long long *counters;     // [4] or null
    uint32_t *mask;                   // trace: [n*H*W][words]
    int32_t *nlat;                    // trace: [n*H*W]
    int words;
    int W, H, cam0;
    float step, t_term;
    int early_term;
    int contraction;                  // 0: contract_pi (Sec. 3.2); 1: spherical ablation, dense
    CamBlock cams;
};

__device__ __forceinline__ float sigmoid_f(float x) { return __fdividef(1.0f, 1.0f + __expf(-x)); }

// 2^x and 1/x by the special-function unit (PTX ex2.approx / rcp.approx, relative error about
// 2^-22): sigmoid(x) = 1 / (1 + 2^y) with y = -x log2(e).
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
constexpr float kLog2e = 1.44269504088896341f;

// Appearance of one sample as exponents y = -x log2(e) of its seven sigmoids: channel 1 and
// the pairs (2, 3), (4, 5), (6, 7), so that pairs go through packed FP32 arithmetic.
struct AppArg {
    float y1;
    float2 y23, y45, y67;
};

__device__ __forceinline__ AppArg app_arg(const float app[7])
{
    const float2 nl = make_float2(-kLog2e, -kLog2e);
    AppArg a;
    a.y1 = app[0] * -kLog2e;
    a.y23 = __fmul2_rn(make_float2(app[1], app[2]), nl);
    a.y45 = __fmul2_rn(make_float2(app[3], app[4]), nl);
    a.y67 = __fmul2_rn(make_float2(app[5], app[6]), nl);
    return a;
}

// From the two-level integer sums of the FP32 uint8 path: x = (14 / 255) K - 7 W (W the sources'
// total weight, as in dequant_density) with K = (256 H + L) / S, so
// y = -x log2(e) = L A / S + (H 256 A / S + 7 log2(e) W), A = -14 log2(e) / 255: two fused
// multiply-adds per channel, in pairs.
__device__ __forceinline__ float2 u2f2(uint32_t a, uint32_t b)
{
    return make_float2(__uint2float_rn(a), __uint2float_rn(b));
}

__device__ __forceinline__ AppArg app_arg_u8(const DotSums<0> &k, float wsum)
{
    const float A = -kLog2e * 14.0f / 255.0f, b = (7.0f * kLog2e) * wsum;
    const float Al = A * (1.0f / kWScale), Ah = A * (256.0f / kWScale);
    const float2 Al2 = make_float2(Al, Al), Ah2 = make_float2(Ah, Ah), b2 = make_float2(b, b);
    AppArg a;
    a.y1 = fmaf(__uint2float_rn(k.lo[1]), Al, fmaf(__uint2float_rn(k.hi[1]), Ah, b));
    a.y23 = __ffma2_rn(u2f2(k.lo[2], k.lo[3]), Al2, __ffma2_rn(u2f2(k.hi[2], k.hi[3]), Ah2, b2));
    a.y45 = __ffma2_rn(u2f2(k.lo[4], k.lo[5]), Al2, __ffma2_rn(u2f2(k.hi[4], k.hi[5]), Ah2, b2));
    a.y67 = __ffma2_rn(u2f2(k.lo[6], k.lo[7]), Al2, __ffma2_rn(u2f2(k.hi[6], k.hi[7]), Ah2, b2));
    return a;
}

// Front-to-back accumulators of C_d (channels 1..3) and F (channels 4..7), paired as AppArg.
struct Accum {
    float c0;
    float2 c12, f01, f23;
};

__device__ __forceinline__ float2 sigmoid2(float2 y)
{
    const float2 e = __fadd2_rn(make_float2(ex2_approx(y.x), ex2_approx(y.y)), make_float2(1.0f, 1.0f));
    return make_float2(rcp_approx(e.x), rcp_approx(e.y));
}

// acc += w sigmoid(x) for the seven appearance channels (Eq. 4 with weight w = alpha T).
__device__ __forceinline__ void composite(Accum &acc, float w, const AppArg &a)
{
    const float2 w2 = make_float2(w, w);
    acc.c0 = fmaf(w, rcp_approx(1.0f + ex2_approx(a.y1)), acc.c0);
    acc.c12 = __ffma2_rn(w2, sigmoid2(a.y23), acc.c12);
    acc.f01 = __ffma2_rn(w2, sigmoid2(a.y45), acc.f01);
    acc.f23 = __ffma2_rn(w2, sigmoid2(a.y67), acc.f23);
}

__device__ __forceinline__ float tanh_approx(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 16-bit forms: sigmoid(x) = (1 + tanh(x / 2)) / 2, so AppArg holds t = x / 2 =
// (7 / 255) K - 3.5 W with the rounded high-level sums K = H' / 32767, and compositing
// accumulates only (w / 2) tanh(t); the constant halves sum to (1 - T) / 2 per ray (the weights
// alpha_i T_i sum to 1 - T), added once at the end.
template <int kPrec>
__device__ __forceinline__ AppArg app_arg_u8_half(const DotSums<kPrec> &k, float wsum)
{
    const float A = 7.0f / 255.0f * (256.0f / kWScale), b = -3.5f * wsum;
    const float2 A2 = make_float2(A, A), b2 = make_float2(b, b);
    AppArg a;
    a.y1 = fmaf(__uint2float_rn(k.hi[1]), A, b);
    a.y23 = __ffma2_rn(u2f2(k.hi[2], k.hi[3]), A2, b2);
    a.y45 = __ffma2_rn(u2f2(k.hi[4], k.hi[5]), A2, b2);
    a.y67 = __ffma2_rn(u2f2(k.hi[6], k.hi[7]), A2, b2);
    return a;
}

__device__ __forceinline__ void composite_tanh(Accum &acc, float w, const AppArg &a)
{
    const float hw = 0.5f * w;
    const float2 hw2 = make_float2(hw, hw);
    acc.c0 = fmaf(hw, tanh_approx(a.y1), acc.c0);
    acc.c12 = __ffma2_rn(hw2, make_float2(tanh_approx(a.y23.x), tanh_approx(a.y23.y)), acc.c12);
    acc.f01 = __ffma2_rn(hw2, make_float2(tanh_approx(a.y45.x), tanh_approx(a.y45.y)), acc.f01);
    acc.f23 = __ffma2_rn(hw2, make_float2(tanh_approx(a.y67.x), tanh_approx(a.y67.y)), acc.f23);
}

// gamma(d) into x[10 .. 33]: sin and cos of 2^l d_k for l = 0..3 (App. B), at x[10 + 6 l + k] and
// x[13 + 6 l + k].  The base frequency comes from sincosf; each doubled one from the previous by
// sin 2a = (2 sin a) cos a and cos 2a = 1 - (2 sin a) sin a, one rounding each (2 sin a is exact).
// A doubling about doubles the absolute error it inherits, which stays near 1e-6 after three.
__device__ __forceinline__ void posenc(const float d[3], float *x)
{
#pragma unroll
    for (int k = 0; k < 3; ++k) sincosf(d[k], &x[10 + k], &x[13 + k]);
#pragma unroll
    for (int l = 1; l < 4; ++l)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float s2 = 2.0f * x[10 + 6 * (l - 1) + k], c = x[13 + 6 * (l - 1) + k];
            x[10 + 6 * l + k] = s2 * c;
            x[13 + 6 * l + k] = fmaf(-s2, x[10 + 6 * (l - 1) + k], 1.0f);
        }
}

// h(C_d, F, d): [C_d, F, d, sin d, cos d, sin 2d, cos 2d, sin 4d, cos 4d, sin 8d, cos 8d]
// -> 16 ReLU -> 16 ReLU -> 3 (App. B: three layers, 16 hidden units, 4 frequencies).  The 16-wide
// layers run as packed FP32 pairs over the outputs (each lane rounds as fmaf does), with the
// weights read 4 at a time from shared memory (w 16-byte aligned).
__device__ __forceinline__ void mlp_f32(const float *w, const float cd[3], const float f[4],
                                        const float d[3], float out[3])
{
    const float4 *W0 = reinterpret_cast<const float4 *>(w), *b0 = reinterpret_cast<const float4 *>(w + 544);
    const float4 *W1 = reinterpret_cast<const float4 *>(w + 560), *b1 = reinterpret_cast<const float4 *>(w + 816);
    const float *W2 = w + 832, *b2 = w + 880;
    float2 h1[8], h2[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 b = b0[q];
        h1[2 * q] = make_float2(b.x, b.y);
        h1[2 * q + 1] = make_float2(b.z, b.w);
    }
    // layer 1, input row i of W0 times x_i; the encoding is produced level by level (as posenc
    // does, same values, same row order) so that only one level's sines and cosines are live
    auto row = [&](int i, float xi) {
        const float2 x2 = make_float2(xi, xi);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 wq = W0[i * 4 + q];
            h1[2 * q] = __ffma2_rn(x2, make_float2(wq.x, wq.y), h1[2 * q]);
            h1[2 * q + 1] = __ffma2_rn(x2, make_float2(wq.z, wq.w), h1[2 * q + 1]);
        }
    };
    row(0, cd[0]); row(1, cd[1]); row(2, cd[2]);
    row(3, f[0]); row(4, f[1]); row(5, f[2]); row(6, f[3]);
    row(7, d[0]); row(8, d[1]); row(9, d[2]);
    float sn[3], cs[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) sincosf(d[k], &sn[k], &cs[k]);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
#pragma unroll
        for (int k = 0; k < 3; ++k) row(10 + 6 * l + k, sn[k]);
#pragma unroll
        for (int k = 0; k < 3; ++k) row(13 + 6 * l + k, cs[k]);
        if (l < 3) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float s2 = 2.0f * sn[k], c = cs[k];
                cs[k] = fmaf(-s2, sn[k], 1.0f);      // cos 2a = 1 - (2 sin a) sin a
                sn[k] = s2 * c;                      // sin 2a = (2 sin a) cos a
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) h1[q] = make_float2(fmaxf(h1[q].x, 0.0f), fmaxf(h1[q].y, 0.0f));
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 b = b1[q];
        h2[2 * q] = make_float2(b.x, b.y);
        h2[2 * q + 1] = make_float2(b.z, b.w);
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const float a = (i & 1) ? h1[i >> 1].y : h1[i >> 1].x;
        const float2 hi = make_float2(a, a);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 wq = W1[i * 4 + q];
            h2[2 * q] = __ffma2_rn(hi, make_float2(wq.x, wq.y), h2[2 * q]);
            h2[2 * q + 1] = __ffma2_rn(hi, make_float2(wq.z, wq.w), h2[2 * q + 1]);
        }
    }
#pragma unroll
    for (int o = 0; o < 3; ++o) out[o] = b2[o];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const float h = fmaxf((i & 1) ? h2[i >> 1].y : h2[i >> 1].x, 0.0f);
#pragma unroll
        for (int o = 0; o < 3; ++o) out[o] = fmaf(h, W2[i * 3 + o], out[o]);
    }
}

// ---------------------------------------------------------------------------------------------
// The deferred MLP on the tensor cores (precision form): the CTA's 128 pixels are one M = 128
// tile of tcgen05.mma (kind::f16: FP16 or BF16 operands, FP32 accumulator in tensor memory).
// Layer 1 is [128 x 48] x [48 x 16] (34 inputs zero-padded to 48, three K = 16 steps), layer 2
// [128 x 16] x [16 x 16], layer 3 [128 x 16] x [16 x 16] (3 outputs zero-padded to 16).  The A
// operand (the pixels' activations) is staged in tensor memory: every thread writes its own pixel's
// row into its TMEM lane with tcgen05.st, so the operand takes no shared memory (which the gathers
// use as L1 cache) and needs no layout beyond "row per lane".  The B operand (the weights) sits in
// shared memory.  One thread issues each layer's MMAs and commits them to an mbarrier; every thread
// then reads its own pixel's row of the accumulator (TMEM lane = pixel), adds the bias, applies
// ReLU and writes its row of the next layer's A operand.  BF16 keeps only 8 significant bits, so in
// that mode every operand is carried as an unevaluated sum hi + lo of two bfloat16 values and each
// product takes three passes (hi*hi + lo*hi + hi*lo, all accumulated in FP32); FP16 uses one.

// Tensor-memory columns of a CTA: the accumulator (16), layer 1's A operand (48 halves in 24
// columns) and, for BF16, its low parts (24); layers 2 and 3 reuse the first 8 (+ 8) A columns.
constexpr int kTmemCols = 64;
constexpr int kColD = 0, kColA = 16, kColALo = 40;
// Bounded waits (an MMA group or the weights' bulk copy completes in microseconds): 2 ms of the
// global timer, after which the wait gives up and the status word records it.
constexpr uint32_t kWaitNs = 2000000;

// The weights of one 16-bit form as the MMAs read them, built once per scene in device memory and
// brought to shared memory by one bulk copy: the B operands W0^T, W1^T, W2^T as K-major 16-bit
// tiles (each with its BF16 low part in [1]), then the FP32 biases.
template <int kPrec>
struct alignas(128) MlpWeights16 {
    static constexpr int kParts = kPrec == 2 ? 2 : 1;     // [1]: BF16 low parts
    uint8_t w0[kParts][16 * 48 * 2];                       // W0^T [n][k], k >= 34 zero
    uint8_t w1[kParts][16 * 16 * 2];                       // W1^T
    uint8_t w2[kParts][16 * 16 * 2];                       // W2^T, rows n >= 3 zero
    float b0[16], b1[16], b2[4];                           // b2[3] zero
};

template <int kPrec>
struct MlpUmma {
    static constexpr int kParts = MlpWeights16<kPrec>::kParts;
    MlpWeights16<kPrec> wt;
    alignas(8) uint64_t mbar;                              // MMA completion
    uint32_t tmem;                                         // the CTA's tensor-memory columns
};

// Per-thread state of the CTA's rounds: the completion barrier's next parity, and whether every
// round so far completed (after a round that did not, no further MMA is issued, and the CTA waits
// once more for that round before it frees its tensor memory).
struct UmmaState {
    uint32_t phase = 0, failed_parity = 0;
    bool ok = true;
};

// A scene's MLP block in device memory: the 883 FP32 weights padded to 884 (16 bytes), then the
// FP16 and the BF16 forms, each at a 128-byte boundary.  Each form is one bulk copy: 16-byte
// aligned at both ends and a multiple of 16 bytes long.
constexpr int kMlpF32Floats = 884;
constexpr size_t kMlpOffF16 = 3584;
constexpr size_t kMlpOffBf16 = kMlpOffF16 + sizeof(MlpWeights16<1>);
constexpr size_t kMlpBlockBytes = kMlpOffBf16 + sizeof(MlpWeights16<2>);
static_assert(kMlpF32Floats >= kMlpParams && kMlpF32Floats * 4 % 16 == 0 && kMlpF32Floats * 4 <= kMlpOffF16,
              "FP32 form: one 16-byte multiple before the FP16 form");
static_assert(kMlpOffF16 % 128 == 0 && kMlpOffBf16 % 128 == 0, "forms at 128-byte boundaries");
static_assert(sizeof(MlpWeights16<1>) % 16 == 0 && sizeof(MlpWeights16<2>) % 16 == 0, "bulk-copy sizes");

template <int kPrec>
__host__ __device__ constexpr size_t mlp_form_offset()
{
    return kPrec == 0 ? 0 : kPrec == 1 ? kMlpOffF16 : kMlpOffBf16;
}

template <int kPrec>
__device__ __forceinline__ uint32_t pack16(float lo, float hi)
{
    uint32_t u;
    if constexpr (kPrec == 1) {
        const __half2 h = __floats2half2_rn(lo, hi);
        memcpy(&u, &h, 4);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        memcpy(&u, &h, 4);
    }
    return u;
}

// low part of a BF16 split: lo = bf16(v - float(bf16(v)))
__device__ __forceinline__ float bf16_rest(float v)
{
    return v - __bfloat162float(__float2bfloat16_rn(v));
}

template <int kPrec>
__device__ __forceinline__ uint32_t pack16_lo(float lo, float hi)
{
    return pack16<kPrec>(bf16_rest(lo), bf16_rest(hi));
}

// One 16-bit element pair (k, k + 1) of row n of a K-major B tile, with its BF16 low part.
template <int kPrec, int K, int kBytes>
__device__ __forceinline__ void put_w(uint8_t (&w)[MlpWeights16<kPrec>::kParts][kBytes], int n, int k, float a, float b)
{
    const int off = kmajor_offset(n, k, K);
    *reinterpret_cast<uint32_t *>(&w[0][off]) = pack16<kPrec>(a, b);
    if constexpr (kPrec == 2) *reinterpret_cast<uint32_t *>(&w[1][off]) = pack16_lo<kPrec>(a, b);
}

// TMEM columns and the completion barrier (before the CTA's first barrier).
template <int kPrec>
__device__ __forceinline__ void mlp_umma_init(MlpUmma<kPrec> &ms)
{
    if (threadIdx.x < 32) tmem_alloc<kTmemCols>(&ms.tmem);
    if (threadIdx.x == 0) {
        mbar_init(&ms.mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
}

// Every warp's accumulator reads are done; warp 0 frees the columns (all threads call it).  If a
// round did not complete, its MMAs may still be running: wait for them once more (bounded) first.
template <int kPrec>
__device__ __forceinline__ void mlp_umma_fini(MlpUmma<kPrec> &ms, const UmmaState &us)
{
    tc_fence_before();
    const bool ok = __syncthreads_and(us.ok);
    if (!ok) mbar_wait(&ms.mbar, us.failed_parity, kWaitNs);
    if (threadIdx.x < 32) {
        tc_fence_after();
        tmem_dealloc<kTmemCols>(ms.tmem);
    }
}

// Pack the FP32 weights w (layout of App. B: W0 [34][16], b0, W1 [16][16], b1, W2 [16][3], b2)
// into one 16-bit form (the threads of one CTA).
template <int kPrec>
__device__ __forceinline__ void mlp_pack16(MlpWeights16<kPrec> &o, const float *w)
{
    const float *W0 = w, *B0 = w + 544, *W1 = w + 560, *B1 = w + 816, *W2 = w + 832, *B2 = w + 880;
    for (int e = threadIdx.x; e < 16 * 24; e += kThreads) {
        const int n = e / 24, k = 2 * (e % 24);
        const float a = k < 34 ? __ldg(W0 + k * 16 + n) : 0.0f;
        const float b = k + 1 < 34 ? __ldg(W0 + (k + 1) * 16 + n) : 0.0f;
        put_w<kPrec, 48>(o.w0, n, k, a, b);
    }
    for (int e = threadIdx.x; e < 16 * 8; e += kThreads) {
        const int n = e / 8, k = 2 * (e % 8);
        put_w<kPrec, 16>(o.w1, n, k, __ldg(W1 + k * 16 + n), __ldg(W1 + (k + 1) * 16 + n));
        const float a = n < 3 ? __ldg(W2 + k * 3 + n) : 0.0f, b = n < 3 ? __ldg(W2 + (k + 1) * 3 + n) : 0.0f;
        put_w<kPrec, 16>(o.w2, n, k, a, b);
    }
    for (int e = threadIdx.x; e < 16; e += kThreads) {
        o.b0[e] = __ldg(B0 + e);
        o.b1[e] = __ldg(B1 + e);
        if (e < 4) o.b2[e] = e < 3 ? __ldg(B2 + e) : 0.0f;
    }
}

// This thread's row (pixel) of a K-column A operand into its TMEM lane from column `col` (BF16
// low parts if kLow): two 16-bit elements per column, 8 columns per store.
template <int kPrec, int K, bool kLow>
__device__ __forceinline__ void put_row(uint32_t tmem, int col, const float *v)
{
#pragma unroll
    for (int c = 0; c < K / 16; ++c) {
        uint32_t u[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            u[q] = kLow ? pack16_lo<kPrec>(v[16 * c + 2 * q], v[16 * c + 2 * q + 1])
                        : pack16<kPrec>(v[16 * c + 2 * q], v[16 * c + 2 * q + 1]);
        tmem_st8(tmem, col + 8 * c, u);
    }
}

// D (+)= A B over K (K / 16 MMAs of K = 16: 8 TMEM columns of A, two 128-byte core-matrix columns
// of B each), A in TMEM from column a, B a K-major tile at shared address b.  Issuing thread only.
template <int kPrec, int K>
__device__ __forceinline__ void mma_k(uint32_t tmem, uint32_t a, uint32_t b, bool accumulate)
{
    constexpr uint32_t kId = umma_idesc_f16(128, 16, kPrec == 2), kSbo = (K / 8) * 128;
#pragma unroll
    for (int ks = 0; ks < K / 16; ++ks)
        umma_f16_ts(tmem + kColD, a + 8u * ks, umma_smem_desc(b + 256u * ks, 128, kSbo), kId, accumulate || ks > 0);
}

// One round on the tensor cores: every thread's operand rows are published, thread 0 issues the
// MMAs (`issue`) and commits them to the barrier, and all threads wait for them.  False if this
// round's wait gave up (recorded in the device status word; uniform within each warp) or an
// earlier one did (uniform across the CTA: then nothing is issued).
template <int kPrec, typename Issue>
__device__ __forceinline__ bool umma_round(MlpUmma<kPrec> &ms, UmmaState &us, Issue issue)
{
    tmem_st_wait();              // this thread's operand rows are in tensor memory
    tc_fence_before();
    us.ok = __syncthreads_and(us.ok);   // all rows written; every earlier accumulator read done
    tc_fence_after();
    if (!us.ok) return false;
    if (threadIdx.x == 0) {
        issue();
        umma_commit(&ms.mbar);
    }
    const bool done = __all_sync(0xffffffffu, mbar_wait(&ms.mbar, us.phase, kWaitNs));
    if (!done) {
        us.ok = false;
        us.failed_parity = us.phase;
        if ((threadIdx.x & 31) == 0) set_status(kWaitTimeout);
    }
    us.phase ^= 1u;
    tc_fence_after();
    return done;
}

// This thread's accumulator row (nc = 16 or 4 columns), zeros if the MMAs did not complete.
template <int nc>
__device__ __forceinline__ void acc_row(uint32_t tmem, bool ok, float *acc)
{
    if (ok) {
        if constexpr (nc == 16) tmem_ld16(tmem, 0, acc);
        else tmem_ld4(tmem, 0, acc);
    } else {
#pragma unroll
        for (int c = 0; c < nc; ++c) acc[c] = 0.0f;
    }
}

// A 16-input layer (2 or 3): D = H W, BF16 as hi*hi + lo*hi + hi*lo in one round.
template <int kPrec, int nc>
__device__ __forceinline__ void layer16(MlpUmma<kPrec> &ms, UmmaState &us, uint8_t (&w)[MlpWeights16<kPrec>::kParts][512],
                                        const float h[16], float *acc)
{
    const uint32_t tm = ms.tmem;
    put_row<kPrec, 16, false>(tm, kColA, h);
    if constexpr (kPrec == 2) put_row<kPrec, 16, true>(tm, kColALo, h);
    const uint32_t wh = smem_addr(w[0]), wl = smem_addr(w[MlpUmma<kPrec>::kParts - 1]);
    const bool ok = umma_round(ms, us, [&] {
        mma_k<kPrec, 16>(tm, tm + kColA, wh, false);
        if constexpr (kPrec == 2) {
            mma_k<kPrec, 16>(tm, tm + kColALo, wh, true);
            mma_k<kPrec, 16>(tm, tm + kColA, wl, true);
        }
    });
    acc_row<nc>(tm + kColD, ok, acc);
}

// h(C_d, F, d) of this thread's pixel; all 128 threads of the CTA call it together (threads
// without a pixel pass zeros and ignore the result).
template <int kPrec>
__device__ __forceinline__ void mlp_umma(MlpUmma<kPrec> &ms, UmmaState &us, const float cd[3], const float f[4],
                                         const float d[3], float out[3])
{
    float x[48];
    x[0] = cd[0]; x[1] = cd[1]; x[2] = cd[2];
    x[3] = f[0]; x[4] = f[1]; x[5] = f[2]; x[6] = f[3];
    x[7] = d[0]; x[8] = d[1]; x[9] = d[2];
    posenc(d, x);
#pragma unroll
    for (int k = 34; k < 48; ++k) x[k] = 0.0f;
    // layer 1 (BF16: hi*hi + hi*lo + lo*hi, the low parts in their own columns)
    const uint32_t tm = ms.tmem, wh = smem_addr(ms.wt.w0[0]), wl = smem_addr(ms.wt.w0[MlpUmma<kPrec>::kParts - 1]);
    put_row<kPrec, 48, false>(tm, kColA, x);
    if constexpr (kPrec == 2) put_row<kPrec, 48, true>(tm, kColALo, x);
    const bool ok = umma_round(ms, us, [&] {
        mma_k<kPrec, 48>(tm, tm + kColA, wh, false);
        if constexpr (kPrec == 2) {
            mma_k<kPrec, 48>(tm, tm + kColA, wl, true);
            mma_k<kPrec, 48>(tm, tm + kColALo, wh, true);
        }
    });
    float h[16];
    acc_row<16>(tm + kColD, ok, h);
#pragma unroll
    for (int o = 0; o < 16; ++o) h[o] = fmaxf(h[o] + ms.wt.b0[o], 0.0f);
    float h2[16];
    layer16<kPrec, 16>(ms, us, ms.wt.w1, h, h2);
#pragma unroll
    for (int o = 0; o < 16; ++o) h2[o] = fmaxf(h2[o] + ms.wt.b1[o], 0.0f);
    float y[4];
    layer16<kPrec, 4>(ms, us, ms.wt.w2, h2, y);
    out[0] = y[0] + ms.wt.b2[0];
    out[1] = y[1] + ms.wt.b2[1];
    out[2] = y[2] + ms.wt.b2[2];
}

__device__ __forceinline__ void pixel_of_thread(int &i, int &j)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    i = blockIdx.x * kTileW + (warp & 1) * 8 + (lane & 7);
    j = blockIdx.y * kTileH + (warp >> 1) * 4 + (lane >> 3);
}

// Result of marching one ray (before the deferred MLP).
struct RayState {
    float cd[3], F[4], T, d[3];
    int nlat, neval, napp, term;
};

// March one pixel ray: traversal, gather, activations and front-to-back compositing.
// Pre-activation density and appearance exponents of the field at a contracted point: all
// channels in one tap-major pass; the appearance values are used only when the opacity is
// non-zero (Sec. 5), which changes nothing else (weight alpha T = 0).
template <int kStorage, int kPrec, int kGeo>
__device__ __forceinline__ void eval_field(const FieldView &fv, float p0, float p1, float p2, float &dens, AppArg &ya)
{
    if constexpr (kStorage == 0) {
        Taps tp;
        gather_u8<kGeo>(fv, p0, p1, p2, tp);
        DotSums<kPrec> k;
        dot_sums<kPrec, kTaps<kGeo>>(tp, k);      // 16-bit forms: appearance at one level
        const float wsum = tp.wv + (float)kPlaneSources<kGeo>;
        dens = dequant_density<kPrec>(k, wsum);
        if constexpr (kPrec == 0) ya = app_arg_u8(k, wsum);
        else ya = app_arg_u8_half<kPrec>(k, wsum);
    } else {
        float all[8];
        field_f32<kGeo>(fv, p0, p1, p2, all);
        dens = all[0];
        ya = app_arg(all + 1);
    }
}

// March one pixel ray: traversal, gather, activations and front-to-back compositing.
template <int kStorage, int kPrec, int kGeo = kGeoRuntime>
__device__ __forceinline__ void march_ray(const FieldView &fv, const OccView &occ, const float *cam, int i, int j,
                                          float step, float t_term, int early_term, RayState &r)
{
    float o[3];
    ray_f32(cam, i, j, o, r.d);
    Walker wk;
    wk.init(o, r.d, step);
    r.nlat = wk.nlat;
    Accum acc;
    acc.c0 = 0.0f;
    acc.c12 = acc.f01 = acc.f23 = make_float2(0.0f, 0.0f);
    for (;;) {
        float p0, p1, p2;
        if (!wk.next_sample<typename GatherIndex<kGeo>::T>(occ, p0, p1, p2)) break;
        float dens;
        AppArg ya;
        eval_field<kStorage, kPrec, kGeo>(fv, p0, p1, p2, dens, ya);
        const float tau = __expf(dens);
        const float dw = wk.delta_world(wk.k);
        const float alpha = 1.0f - __expf(-tau * dw);
        ++r.neval;
        if (alpha > 0.0f) {
            ++r.napp;
            if constexpr (kPrec == 0) composite(acc, alpha * r.T, ya);
            else composite_tanh(acc, alpha * r.T, ya);
            r.T = r.T * (1.0f - alpha);
            if (early_term && r.T < t_term) { r.term = 1; break; }
        }
        ++wk.k;
    }
    if constexpr (kPrec != 0) {
        const float h = 0.5f * (1.0f - r.T);
        acc.c0 += h;
        acc.c12 = __fadd2_rn(acc.c12, make_float2(h, h));
        acc.f01 = __fadd2_rn(acc.f01, make_float2(h, h));
        acc.f23 = __fadd2_rn(acc.f23, make_float2(h, h));
    }
    r.cd[0] = acc.c0; r.cd[1] = acc.c12.x; r.cd[2] = acc.c12.y;
    r.F[0] = acc.f01.x; r.F[1] = acc.f01.y; r.F[2] = acc.f23.x; r.F[3] = acc.f23.y;
}

// The spherical-contraction ablation: the same field, quadrature and compositing, with every
// sample of the dense march visited and its own finest occupancy cell tested (no skipping).
template <int kStorage, int kGeo>
__device__ __forceinline__ void march_ray_sph(const FieldView &fv, const OccView &occ, const float *cam, int i,
                                              int j, float step, float t_term, int early_term, RayState &r)
{
    float o[3];
    ray_f32(cam, i, j, o, r.d);
    const int n = sph_count(step);
    r.nlat = n;
    Accum acc;
    acc.c0 = 0.0f;
    acc.c12 = acc.f01 = acc.f23 = make_float2(0.0f, 0.0f);
    const int N0 = occ.res[0];
    const float sc0 = (float)N0 * 0.25f;
    const int h0 = N0 >> 1;
    for (int k = 0; k < n; ++k) {
        float p[3];
        sph_point(o, r.d, step, k, p);
        const int c0 = cell_of(p[0], sc0, h0, N0), c1 = cell_of(p[1], sc0, h0, N0), c2 = cell_of(p[2], sc0, h0, N0);
        const size_t oi = ((size_t)c2 * N0 + c1) * N0 + c0;
        if (!MERF_IN_RANGE(oi, (long long)N0 * N0 * N0, kBadOcc) || __ldg(occ.level[0] + oi) == 0) continue;
        float dens;
        AppArg ya;
        eval_field<kStorage, 0, kGeo>(fv, p[0], p[1], p[2], dens, ya);
        const float tau = __expf(dens);
        const float dw = sph_t(F_MUL(F_ADD((float)k, 1.0f), step)) - sph_t(F_MUL((float)k, step));
        const float alpha = 1.0f - __expf(-tau * dw);
        ++r.neval;
        if (alpha > 0.0f) {
            ++r.napp;
            composite(acc, alpha * r.T, ya);
            r.T = r.T * (1.0f - alpha);
            if (early_term && r.T < t_term) { r.term = 1; break; }
        }
    }
    r.cd[0] = acc.c0; r.cd[1] = acc.c12.x; r.cd[2] = acc.c12.y;
    r.F[0] = acc.f01.x; r.F[1] = acc.f01.y; r.F[2] = acc.f23.x; r.F[3] = acc.f23.y;
}

__device__ __forceinline__ void ray_state_init(RayState &r)
{
    r.cd[0] = r.cd[1] = r.cd[2] = 0.0f;
    r.F[0] = r.F[1] = r.F[2] = r.F[3] = 0.0f;
    r.T = 1.0f;
    r.d[0] = 0.0f; r.d[1] = 0.0f; r.d[2] = 1.0f;
    r.nlat = r.neval = r.napp = r.term = 0;
}

// Shared-memory weights of the deferred MLP for one precision, staged by one bulk (TMA) copy of
// the form from the scene's MLP block.  Thread 0 issues the copy (fetch) when the CTA starts or
// changes scene; it lands while the rays march, and every thread waits for it (wait) just before
// the MLP.  Each fetch completes one phase of `wbar`.
template <int kPrec>
struct MlpStage {
    alignas(8) uint64_t wbar;
    __device__ __forceinline__ void init_bar()
    {
        if (threadIdx.x == 0) {
            mbar_init(&wbar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    // Thread 0; every thread's earlier reads of the destination are ordered before it by a barrier.
    __device__ __forceinline__ void copy(void *dst, const float *mlp, uint32_t bytes)
    {
        if (threadIdx.x == 0) {
            fence_async_smem();
            bulk_g2s(dst, reinterpret_cast<const char *>(mlp) + mlp_form_offset<kPrec>(), bytes, &wbar);
        }
    }
    // All threads; true when the copy has landed (as this thread sees it).  A wait that gives up is
    // recorded in the device status word, and its parity in this thread's `lost` bits.
    __device__ __forceinline__ bool wait(uint32_t &wphase, uint32_t &lost)
    {
        const bool landed = mbar_wait(&wbar, wphase, kWaitNs);
        if (!landed) {
            set_status(kWaitTimeout);
            lost |= 1u << wphase;           // bit p: a copy completing parity p is outstanding
        }
        wphase ^= 1u;
        return landed;
    }
    // All threads, before the CTA exits: a copy whose wait gave up may still be in flight into this
    // CTA's shared memory; wait for it once more (bounded).
    __device__ __forceinline__ void drain(uint32_t lost)
    {
        if (lost & 1u) mbar_wait(&wbar, 0, kWaitNs);
        if (lost & 2u) mbar_wait(&wbar, 1, kWaitNs);
    }
};

template <int kPrec>
struct MlpSmem;
template <>
struct MlpSmem<0> : MlpStage<0> {
    alignas(16) float w[kMlpF32Floats];
    __device__ __forceinline__ void init() { init_bar(); }                       // before a barrier
    __device__ __forceinline__ void fetch(const float *mlp) { copy(w, mlp, sizeof w); }
    __device__ __forceinline__ void fini(const UmmaState &, uint32_t lost) { drain(lost); }
};
template <int kPrec>
struct MlpSmem : MlpStage<kPrec> {
    MlpUmma<kPrec> tc;
    __device__ __forceinline__ void init()                                       // before a barrier
    {
        this->init_bar();
        mlp_umma_init<kPrec>(tc);
    }
    __device__ __forceinline__ void fetch(const float *mlp) { this->copy(&tc.wt, mlp, sizeof tc.wt); }
    __device__ __forceinline__ void fini(const UmmaState &us, uint32_t lost)   // all threads, at the end
    {
        this->drain(lost);
        mlp_umma_fini<kPrec>(tc, us);
    }
};

// h(C_d, F, d) for this thread's pixel (every thread of the CTA calls; `live` ones own a pixel).
// `us`: the tensor-core rounds' state, carried across calls.
template <int kPrec>
__device__ __forceinline__ void deferred_mlp(MlpSmem<kPrec> &ms, UmmaState &us, const RayState &r, bool live,
                                             float h[3])
{
    if constexpr (kPrec == 0) {
        if (live) mlp_f32(ms.w, r.cd, r.F, r.d, h);
    } else {
        mlp_umma<kPrec>(ms.tc, us, r.cd, r.F, r.d, h);        // whole CTA, tensor cores
    }
}

// Resident CTAs per SM the register allocation is bounded for (measured: the uint8 kernels on
// the 8 x 1080p paper-scale workload and the dense float kernel on 4 x 512^2 are fastest at 6,
// i.e. 80 registers per thread).
template <int kStorage, int kPrec>
constexpr int kMinBlocks = 6;

template <int kStorage, int kPrec, int kGeo, int kSph = 0>
// storage 0: uint8 block-sparse, 1: float32 dense; precision 0: FP32, 1: FP16, 2: BF16 (uint8
// only); kGeo: gather geometry; kSph 1: the spherical-contraction ablation (FP32)
__global__ void __launch_bounds__(kThreads, (kMinBlocks<kStorage, kPrec>)) render_kernel(const __grid_constant__ RenderParams P)
{
    __shared__ MlpSmem<kPrec> ms;
    ms.init();
    __syncthreads();
    ms.fetch(P.mlp);                   // lands while the rays march

    int i, j;
    pixel_of_thread(i, j);
    const int cl = blockIdx.z;
    const bool inside = (i < P.W) && (j < P.H);
    RayState r;
    ray_state_init(r);
    if (inside) {
        if constexpr (kSph == 0)
            march_ray<kStorage, kPrec, kGeo>(P.fv, P.occ, P.cams.m[cl], i, j, P.step, P.t_term, P.early_term, r);
        else
            march_ray_sph<kStorage, kGeo>(P.fv, P.occ, P.cams.m[cl], i, j, P.step, P.t_term, P.early_term, r);
    }
    float h[3];
    UmmaState us;
    uint32_t wphase = 0, lost = 0;
    ms.wait(wphase, lost);             // a copy that did not land leaves garbage weights and the status bit
    deferred_mlp<kPrec>(ms, us, r, inside, h);
    if (inside) {
        const size_t pix = ((size_t)(P.cam0 + cl) * P.H + j) * P.W + i;
        // streaming stores: the image is not read again by this launch, so it should not
        // displace the scene's texels or the rays' stacks in L2
        __stcs(P.out + pix * 3 + 0, r.cd[0] + h[0]);
        __stcs(P.out + pix * 3 + 1, r.cd[1] + h[1]);
        __stcs(P.out + pix * 3 + 2, r.cd[2] + h[2]);
        if (P.aux) {
            float *a = P.aux + pix * kAuxSize;
            a[0] = r.cd[0]; a[1] = r.cd[1]; a[2] = r.cd[2];
            a[3] = r.F[0]; a[4] = r.F[1]; a[5] = r.F[2]; a[6] = r.F[3];
            a[7] = r.T;
            a[8] = (float)r.nlat; a[9] = (float)r.neval; a[10] = (float)r.napp; a[11] = (float)r.term;
        }
    }
    if (P.counters) {
        unsigned long long cr = inside ? 1ull : 0ull, l = r.nlat, e = r.neval, a = r.napp;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            cr += __shfl_down_sync(0xffffffffu, cr, off);
            l += __shfl_down_sync(0xffffffffu, l, off);
            e += __shfl_down_sync(0xffffffffu, e, off);
            a += __shfl_down_sync(0xffffffffu, a, off);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(P.counters + 0, cr);
            atomicAdd(P.counters + 1, l);
            atomicAdd(P.counters + 2, e);
            atomicAdd(P.counters + 3, a);
        }
    }
    ms.fini(us, lost);
}

// Traversal only (no gather, no termination): the set of evaluated lattice samples per ray.
static __global__ void __launch_bounds__(kThreads) trace_kernel(const __grid_constant__ RenderParams P)
{
    int i, j;
    pixel_of_thread(i, j);
    if (i >= P.W || j >= P.H) return;
    const int cl = blockIdx.z;
    const size_t pix = ((size_t)(P.cam0 + cl) * P.H + j) * P.W + i;
    uint32_t *row = P.mask + pix * P.words;
    for (int w = 0; w < P.words; ++w) row[w] = 0u;
    float o[3], d[3];
    ray_f32(P.cams.m[cl], i, j, o, d);
    if (P.contraction == 1) {          // spherical ablation: every sample of the dense march
        const int n = sph_count(P.step);
        P.nlat[pix] = n;
        const int N0 = P.occ.res[0];
        const float sc0 = (float)N0 * 0.25f;
        const int h0 = N0 >> 1;
        for (int k = 0; k < n && k < 32 * P.words; ++k) {
            float p[3];
            sph_point(o, d, P.step, k, p);
            const int c0 = cell_of(p[0], sc0, h0, N0), c1 = cell_of(p[1], sc0, h0, N0),
                      c2 = cell_of(p[2], sc0, h0, N0);
            const size_t oi = ((size_t)c2 * N0 + c1) * N0 + c0;
            if (MERF_IN_RANGE(oi, (long long)N0 * N0 * N0, kBadOcc) && __ldg(P.occ.level[0] + oi) != 0)
                row[k >> 5] |= 1u << (k & 31);
        }
        return;
    }
    Walker wk;
    wk.init(o, d, P.step);
    P.nlat[pix] = wk.nlat;
    float p0, p1, p2;
    while (wk.next_sample(P.occ, p0, p1, p2)) {
        if (wk.k < 32 * P.words) row[wk.k >> 5] |= 1u << (wk.k & 31);
        ++wk.k;
    }
}

}  // namespace merf
