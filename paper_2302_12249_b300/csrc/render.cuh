// render.cuh -- fused per-ray render kernel and traversal-only kernel for sm_103a.
//
// One thread renders one pixel ray end to end: ray generation, segment table, lattice walk
// with a per-sample finest-cell test and coarse-to-fine empty-space skipping, gather of the 20
// texels of each evaluated sample, all eight channels interpolated in one tap-major pass (the
// appearance values enter the result only when the sample's opacity is non-zero, Sec. 5),
// front-to-back compositing of C_d and F with early termination (Eq. 1, Eq. 2, Sec. 5), and
// finally the deferred MLP h(C_d, F, d) (Sec. 2, App. B), whose 883 weights are staged once per
// CTA in shared memory (FP32: per pixel on the CUDA cores; FP16 / BF16: per warp on the tensor
// cores).  A warp covers an 8 x 4 pixel tile and a CTA a 16 x 8 tile, so neighbouring rays walk
// neighbouring texels together and share L1 lines.  Template parameters select the storage
// (uint8 block-sparse / dense float), the precision (FP32 / FP16 / BF16 appearance arithmetic
// and MLP), the gather geometry (the paper's / grid-only / run-time strides) and the contraction
// (contract_pi, or the spherical ablation's dense march).
#pragma once

#include "field.cuh"
#include "traverse.cuh"

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

// From the weighted byte sums of the uint8 path: x = (14 / 255) k - 7 W (W the sources' total
// weight, as in dequant_density), so y = k (-14 log2(e) / 255) + 7 log2(e) W, one fused
// multiply-add per channel.
__device__ __forceinline__ AppArg app_arg_u8(const float2 k[4], float wsum)
{
    const float A = -kLog2e * 14.0f / 255.0f, b = (7.0f * kLog2e) * wsum;
    const float2 A2 = make_float2(A, A), b2 = make_float2(b, b);
    AppArg a;
    a.y1 = fmaf(k[0].y, A, b);
    a.y23 = __ffma2_rn(k[1], A2, b2);
    a.y45 = __ffma2_rn(k[2], A2, b2);
    a.y67 = __ffma2_rn(k[3], A2, b2);
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

// h(C_d, F, d): [C_d, F, d, sin d, cos d, sin 2d, cos 2d, sin 4d, cos 4d, sin 8d, cos 8d]
// -> 16 ReLU -> 16 ReLU -> 3 (App. B: three layers, 16 hidden units, 4 frequencies).
__device__ __forceinline__ void mlp_f32(const float *w, const float cd[3], const float f[4],
                                        const float d[3], float out[3])
{
    float x[34];
    x[0] = cd[0]; x[1] = cd[1]; x[2] = cd[2];
    x[3] = f[0]; x[4] = f[1]; x[5] = f[2]; x[6] = f[3];
    x[7] = d[0]; x[8] = d[1]; x[9] = d[2];
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const float fr = (float)(1 << l);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float s, c;
            sincosf(fr * d[k], &s, &c);
            x[10 + 6 * l + k] = s;
            x[13 + 6 * l + k] = c;
        }
    }
    const float *W0 = w, *b0 = w + 544, *W1 = w + 560, *b1 = w + 816, *W2 = w + 832, *b2 = w + 880;
    float h1[16], h2[16];
#pragma unroll
    for (int o = 0; o < 16; ++o) h1[o] = b0[o];
#pragma unroll
    for (int i = 0; i < 34; ++i)
#pragma unroll
        for (int o = 0; o < 16; ++o) h1[o] = fmaf(x[i], W0[i * 16 + o], h1[o]);
#pragma unroll
    for (int o = 0; o < 16; ++o) { h1[o] = fmaxf(h1[o], 0.0f); h2[o] = b1[o]; }
#pragma unroll
    for (int i = 0; i < 16; ++i)
#pragma unroll
        for (int o = 0; o < 16; ++o) h2[o] = fmaf(h1[i], W1[i * 16 + o], h2[o]);
#pragma unroll
    for (int o = 0; o < 3; ++o) out[o] = b2[o];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const float h = fmaxf(h2[i], 0.0f);
#pragma unroll
        for (int o = 0; o < 3; ++o) out[o] = fmaf(h, W2[i * 3 + o], out[o]);
    }
}

// ---------------------------------------------------------------------------------------------
// The deferred MLP on tensor cores (precision form): one warp evaluates its 32 pixels with
// mma.sync m16n8k16 (FP16 or BF16 operands, FP32 accumulation).  Layer 1 is [32 x 48] x [48 x 16]
// (34 inputs zero-padded to 48), layer 2 [32 x 16] x [16 x 16], layer 3 [32 x 16] x [16 x 8]
// (3 outputs zero-padded to 8).  A layer's FP32 accumulator fragments, after bias and ReLU, are
// packed directly into the next layer's A fragments (the m16n8 C layout of two adjacent n-tiles
// is the m16k16 A layout), so only the inputs and outputs pass through shared memory.

constexpr int kW0Stride = 28, kW1Stride = 12, kXStride = 28;   // 32-bit words per row (padded)

// BF16 keeps only 8 significant bits, so in that mode every operand is carried as an unevaluated
// sum hi + lo of two bfloat16 values and each product takes three tensor-core passes
// (hi*hi + lo*hi + hi*lo, all accumulated in FP32); FP16 uses one pass.
// Shared memory is kept small (it is carved out of the same on-chip storage as the L1 cache
// that serves the texel gathers): only BF16 stores low parts, and each warp stages the input
// rows of one 16-pixel tile at a time.
template <int kPrec>
struct MlpTC {
    static constexpr int kParts = kPrec == 2 ? 2 : 1;
    uint32_t w0[kParts][16 * kW0Stride];   // W0^T [n][k], k < 48, 16-bit pairs; [1]: BF16 low parts
    uint32_t w1[kParts][16 * kW1Stride];   // W1^T [n][k], k < 16
    uint32_t w2[kParts][8 * kW1Stride];    // W2^T [n][k], n < 3 used
    float b0[16], b1[16], b2[8];
    uint32_t x[kParts][kThreads / 32][16 * kXStride];   // per-warp rows of one tile; [1]: BF16 low parts
};

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

template <int kPrec>
__device__ __forceinline__ void mma16816(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1)
{
    if constexpr (kPrec == 1)
        asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                     "{%0,%1,%2,%3};\n"
                     : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                     : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    else
        asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                     "{%0,%1,%2,%3};\n"
                     : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                     : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Stage the scene's FP32 weights as transposed 16-bit tiles (whole CTA, before a barrier).
template <int kPrec>
__device__ __forceinline__ void mlp_tc_load(MlpTC<kPrec> &ms, const float *w)
{
    const float *W0 = w, *B0 = w + 544, *W1 = w + 560, *B1 = w + 816, *W2 = w + 832, *B2 = w + 880;
    for (int e = threadIdx.x; e < 16 * 24; e += kThreads) {
        const int n = e / 24, kk = 2 * (e % 24);
        const float a = kk < 34 ? __ldg(W0 + kk * 16 + n) : 0.0f;
        const float b = kk + 1 < 34 ? __ldg(W0 + (kk + 1) * 16 + n) : 0.0f;
        ms.w0[0][n * kW0Stride + e % 24] = pack16<kPrec>(a, b);
        if constexpr (kPrec == 2) ms.w0[1][n * kW0Stride + e % 24] = pack16_lo<kPrec>(a, b);
    }
    for (int e = threadIdx.x; e < 16 * 8; e += kThreads) {
        const int n = e / 8, kk = 2 * (e % 8);
        const float a = __ldg(W1 + kk * 16 + n), b = __ldg(W1 + (kk + 1) * 16 + n);
        ms.w1[0][n * kW1Stride + e % 8] = pack16<kPrec>(a, b);
        if constexpr (kPrec == 2) ms.w1[1][n * kW1Stride + e % 8] = pack16_lo<kPrec>(a, b);
    }
    for (int e = threadIdx.x; e < 8 * 8; e += kThreads) {
        const int n = e / 8, kk = 2 * (e % 8);
        const float a = n < 3 ? __ldg(W2 + kk * 3 + n) : 0.0f, b = n < 3 ? __ldg(W2 + (kk + 1) * 3 + n) : 0.0f;
        ms.w2[0][n * kW1Stride + e % 8] = pack16<kPrec>(a, b);
        if constexpr (kPrec == 2) ms.w2[1][n * kW1Stride + e % 8] = pack16_lo<kPrec>(a, b);
    }
    for (int e = threadIdx.x; e < 16; e += kThreads) {
        ms.b0[e] = __ldg(B0 + e);
        ms.b1[e] = __ldg(B1 + e);
        if (e < 8) ms.b2[e] = e < 3 ? __ldg(B2 + e) : 0.0f;
    }
}

template <int kPrec>
__device__ __forceinline__ void relu_pack(const float c0[4], const float c1[4], uint32_t a[4], uint32_t al[4])
{
    const float v[8] = {fmaxf(c0[0], 0.0f), fmaxf(c0[1], 0.0f), fmaxf(c0[2], 0.0f), fmaxf(c0[3], 0.0f),
                        fmaxf(c1[0], 0.0f), fmaxf(c1[1], 0.0f), fmaxf(c1[2], 0.0f), fmaxf(c1[3], 0.0f)};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        a[r] = pack16<kPrec>(v[2 * r], v[2 * r + 1]);
        if (kPrec == 2) al[r] = pack16_lo<kPrec>(v[2 * r], v[2 * r + 1]);
    }
}

// D += A B, with the BF16 split when kPrec == 2 (a/b: high parts, al/bl: low parts)
template <int kPrec>
__device__ __forceinline__ void mma_acc(float d[4], const uint32_t a[4], const uint32_t al[4], uint32_t b0,
                                        uint32_t b1, uint32_t bl0, uint32_t bl1)
{
    mma16816<kPrec>(d, a, b0, b1);
    if constexpr (kPrec == 2) {
        mma16816<kPrec>(d, al, b0, b1);
        mma16816<kPrec>(d, a, bl0, bl1);
    }
}

// All 32 lanes of the warp call this together (lanes without a pixel pass zeros).  The warp's
// pixels form two 16-row tiles (lanes 0-15, 16-31), evaluated one after the other.
template <int kPrec>
__device__ __forceinline__ void mlp_tc(MlpTC<kPrec> &ms, const float cd[3], const float f[4], const float d[3],
                                       float out[3])
{
    constexpr int hi = 0, lo = MlpTC<kPrec>::kParts - 1;
    const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3, row = lane & 15;
    uint32_t *xs = ms.x[hi][threadIdx.x >> 5];
    uint32_t *xl = ms.x[lo][threadIdx.x >> 5];
    float x[48];
    x[0] = cd[0]; x[1] = cd[1]; x[2] = cd[2];
    x[3] = f[0]; x[4] = f[1]; x[5] = f[2]; x[6] = f[3];
    x[7] = d[0]; x[8] = d[1]; x[9] = d[2];
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const float fr = (float)(1 << l);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float sn, cs;
            sincosf(fr * d[k], &sn, &cs);
            x[10 + 6 * l + k] = sn;
            x[13 + 6 * l + k] = cs;
        }
    }
#pragma unroll
    for (int k = 34; k < 48; ++k) x[k] = 0.0f;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        __syncwarp();
        if ((lane >> 4) == t) {
#pragma unroll
            for (int j = 0; j < 24; ++j) {
                xs[row * kXStride + j] = pack16<kPrec>(x[2 * j], x[2 * j + 1]);
                if constexpr (kPrec == 2) xl[row * kXStride + j] = pack16_lo<kPrec>(x[2 * j], x[2 * j + 1]);
            }
        }
        __syncwarp();
        // layer 1: [16 x 48] x [48 x 16]
        float acc[2][4];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            acc[u][0] = acc[u][2] = ms.b0[8 * u + 2 * c];
            acc[u][1] = acc[u][3] = ms.b0[8 * u + 2 * c + 1];
        }
#pragma unroll
        for (int sl = 0; sl < 3; ++sl) {
            const int r0 = g * kXStride + 8 * sl + c, r1 = r0 + 8 * kXStride;
            const uint32_t a[4] = {xs[r0], xs[r1], xs[r0 + 4], xs[r1 + 4]};
            uint32_t al[4] = {0u, 0u, 0u, 0u};
            if constexpr (kPrec == 2) { al[0] = xl[r0]; al[1] = xl[r1]; al[2] = xl[r0 + 4]; al[3] = xl[r1 + 4]; }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int wi = (8 * u + g) * kW0Stride + 8 * sl + c;
                mma_acc<kPrec>(acc[u], a, al, ms.w0[hi][wi], ms.w0[hi][wi + 4], ms.w0[lo][wi], ms.w0[lo][wi + 4]);
            }
        }
        // layer 2: [16 x 16] x [16 x 16]
        float acc2[2][4];
        {
            uint32_t a[4], al[4];
            relu_pack<kPrec>(acc[0], acc[1], a, al);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                acc2[u][0] = acc2[u][2] = ms.b1[8 * u + 2 * c];
                acc2[u][1] = acc2[u][3] = ms.b1[8 * u + 2 * c + 1];
                const int wi = (8 * u + g) * kW1Stride + c;
                mma_acc<kPrec>(acc2[u], a, al, ms.w1[hi][wi], ms.w1[hi][wi + 4], ms.w1[lo][wi], ms.w1[lo][wi + 4]);
            }
        }
        // layer 3: [16 x 16] x [16 x 8]
        float acc3[4];
        {
            uint32_t a[4], al[4];
            relu_pack<kPrec>(acc2[0], acc2[1], a, al);
            acc3[0] = acc3[2] = ms.b2[2 * c];
            acc3[1] = acc3[3] = ms.b2[2 * c + 1];
            const int wi = g * kW1Stride + c;
            mma_acc<kPrec>(acc3, a, al, ms.w2[hi][wi], ms.w2[hi][wi + 4], ms.w2[lo][wi], ms.w2[lo][wi + 4]);
        }
        // the tile's 16 x 3 outputs go back to their pixels through shared memory
        __syncwarp();
        float *os = reinterpret_cast<float *>(xs);
        if (c < 2) {
            os[g * 4 + 2 * c] = acc3[0];
            os[g * 4 + 2 * c + 1] = acc3[1];
            os[(g + 8) * 4 + 2 * c] = acc3[2];
            os[(g + 8) * 4 + 2 * c + 1] = acc3[3];
        }
        __syncwarp();
        if ((lane >> 4) == t) {
            out[0] = os[row * 4 + 0];
            out[1] = os[row * 4 + 1];
            out[2] = os[row * 4 + 2];
        }
    }
    __syncwarp();
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
        float2 k[4];
        if constexpr (kPrec == 0) byte_sums_u8<kTaps<kGeo>>(tp, k);
        else byte_sums_lp<kPrec, kTaps<kGeo>>(tp, k);   // FP16 / BF16 appearance; density FP32
        const float wsum = tp.wv + (float)kPlaneSources<kGeo>;
        dens = dequant_density(k[0].x, wsum);
        ya = app_arg_u8(k, wsum);
    } else {
        float all[8];
        field_f32(fv, p0, p1, p2, all);
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
        if (!wk.next_sample(occ, p0, p1, p2)) break;
        float dens;
        AppArg ya;
        eval_field<kStorage, kPrec, kGeo>(fv, p0, p1, p2, dens, ya);
        const float tau = __expf(dens);
        const float dw = wk.delta_world(wk.k);
        const float alpha = 1.0f - __expf(-tau * dw);
        ++r.neval;
        if (alpha > 0.0f) {
            ++r.napp;
            composite(acc, alpha * r.T, ya);
            r.T = r.T * (1.0f - alpha);
            if (early_term && r.T < t_term) { r.term = 1; break; }
        }
        ++wk.k;
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

// Shared-memory weights of the deferred MLP for one precision.
template <int kPrec>
struct MlpSmem;
template <>
struct MlpSmem<0> {
    float w[kMlpParams];
    __device__ __forceinline__ void load(const float *mlp)
    {
        for (int t = threadIdx.x; t < kMlpParams; t += kThreads) w[t] = __ldg(mlp + t);
    }
};
template <int kPrec>
struct MlpSmem {
    MlpTC<kPrec> tc;
    __device__ __forceinline__ void load(const float *mlp) { mlp_tc_load<kPrec>(tc, mlp); }
};

// h(C_d, F, d) for every thread of the warp (all lanes call; `live` lanes own a pixel).
template <int kPrec>
__device__ __forceinline__ void deferred_mlp(MlpSmem<kPrec> &ms, const RayState &r, bool live, float h[3])
{
    if constexpr (kPrec == 0) {
        if (live) mlp_f32(ms.w, r.cd, r.F, r.d, h);
    } else {
        mlp_tc<kPrec>(ms.tc, r.cd, r.F, r.d, h);     // whole warp, tensor cores
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
    ms.load(P.mlp);
    __syncthreads();

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
    deferred_mlp<kPrec>(ms, r, inside, h);
    if (inside) {
        const size_t pix = ((size_t)(P.cam0 + cl) * P.H + j) * P.W + i;
        P.out[pix * 3 + 0] = r.cd[0] + h[0];
        P.out[pix * 3 + 1] = r.cd[1] + h[1];
        P.out[pix * 3 + 2] = r.cd[2] + h[2];
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
