// render.cuh -- fused per-ray render kernel and traversal-only kernel for sm_103a.
//
// One thread renders one pixel ray end to end: ray generation, segment table, lattice walk
// with coarse-to-fine empty-space skipping (occupied samples come in runs that share a finest
// occupancy cell), gather of the 20 texels of each evaluated sample, density-first activation
// (Sec. 5: appearance is unpacked only when the sample's opacity is non-zero), front-to-back compositing of C_d and F with early termination
// (Eq. 1, Eq. 2, Sec. 5), and finally the deferred MLP h(C_d, F, d) (Sec. 2, App. B), whose
// 883 weights are staged once per CTA in shared memory and read as warp-wide broadcasts.
// A warp covers an 8 x 4 pixel tile and a CTA a 16 x 8 tile, so neighbouring rays walk
// neighbouring texels together and share L1 lines.
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
    CamBlock cams;
};

__device__ __forceinline__ float sigmoid_f(float x) { return __fdividef(1.0f, 1.0f + __expf(-x)); }

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

__device__ __forceinline__ void pixel_of_thread(int &i, int &j)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    i = blockIdx.x * kTileW + (warp & 1) * 8 + (lane & 7);
    j = blockIdx.y * kTileH + (warp >> 1) * 4 + (lane >> 3);
}

template <int kStorage>   // 0: uint8 block-sparse, 1: float32 dense
__global__ void __launch_bounds__(kThreads) render_kernel(const __grid_constant__ RenderParams P)
{
    __shared__ float wsm[kMlpParams];
    for (int t = threadIdx.x; t < kMlpParams; t += kThreads) wsm[t] = __ldg(P.mlp + t);
    __syncthreads();

    int i, j;
    pixel_of_thread(i, j);
    const int cl = blockIdx.z;
    const bool inside = (i < P.W) && (j < P.H);
    int neval = 0, napp = 0, nlat = 0;
    if (inside) {
        const float *cam = P.cams.m[cl];
        float o[3], d[3];
        ray_f32(cam, i, j, o, d);
        Walker wk;
        wk.init(o, d, P.step);
        nlat = wk.nlat;
        float T = 1.0f, cd[3] = {0.0f, 0.0f, 0.0f}, F[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        int term = 0;
        int run_end = 0;
        for (;;) {
            if (wk.k >= run_end && !wk.next_run(P.occ, run_end)) break;
            float p0, p1, p2;
            wk.position(wk.k, p0, p1, p2);
            float dens, app[7];
            Taps tp;
            if (kStorage == 0) {
                gather_u8(P.fv, p0, p1, p2, tp);
                dens = density_u8(tp);
            } else {
                float all[8];
                field_f32(P.fv, p0, p1, p2, all);
                dens = all[0];
#pragma unroll
                for (int c = 0; c < 7; ++c) app[c] = all[1 + c];
            }
            const float tau = __expf(dens);
            const float dw = wk.delta_world(wk.k);
            const float alpha = 1.0f - __expf(-tau * dw);
            ++neval;
            if (alpha > 0.0f) {
                ++napp;
                if (kStorage == 0) appearance_u8(tp, app);
                const float wgt = alpha * T;
#pragma unroll
                for (int c = 0; c < 3; ++c) cd[c] = fmaf(wgt, sigmoid_f(app[c]), cd[c]);
#pragma unroll
                for (int c = 0; c < 4; ++c) F[c] = fmaf(wgt, sigmoid_f(app[3 + c]), F[c]);
                T = T * (1.0f - alpha);
                if (P.early_term && T < P.t_term) { term = 1; break; }
            }
            ++wk.k;
        }
        float h[3];
        mlp_f32(wsm, cd, F, d, h);
        const size_t pix = ((size_t)(P.cam0 + cl) * P.H + j) * P.W + i;
        P.out[pix * 3 + 0] = cd[0] + h[0];
        P.out[pix * 3 + 1] = cd[1] + h[1];
        P.out[pix * 3 + 2] = cd[2] + h[2];
        if (P.aux) {
            float *a = P.aux + pix * kAuxSize;
            a[0] = cd[0]; a[1] = cd[1]; a[2] = cd[2];
            a[3] = F[0]; a[4] = F[1]; a[5] = F[2]; a[6] = F[3];
            a[7] = T;
            a[8] = (float)nlat; a[9] = (float)neval; a[10] = (float)napp; a[11] = (float)term;
        }
    }
    if (P.counters) {
        unsigned long long r = inside ? 1ull : 0ull, l = nlat, e = neval, a = napp;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            r += __shfl_down_sync(0xffffffffu, r, off);
            l += __shfl_down_sync(0xffffffffu, l, off);
            e += __shfl_down_sync(0xffffffffu, e, off);
            a += __shfl_down_sync(0xffffffffu, a, off);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(P.counters + 0, r);
            atomicAdd(P.counters + 1, l);
            atomicAdd(P.counters + 2, e);
            atomicAdd(P.counters + 3, a);
        }
    }
}

// Traversal only (no gather, no termination): the set of evaluated lattice samples per ray.
__global__ void __launch_bounds__(kThreads) trace_kernel(const __grid_constant__ RenderParams P)
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
    Walker wk;
    wk.init(o, d, P.step);
    P.nlat[pix] = wk.nlat;
    int run_end = 0;
    while (wk.next_run(P.occ, run_end)) {
        for (; wk.k < run_end; ++wk.k)
            if (wk.k < 32 * P.words) row[wk.k >> 5] |= 1u << (wk.k & 31);
    }
}

}  // namespace merf
