// backward.cuh -- hand-written adjoint of the renderer for dense float scenes (sm_103a).
//
// For L with dL/dC given per pixel, one thread per ray:
//   1. take C_d, F from the forward pass's per-pixel record, or recompute the forward march
//      (same arithmetic, hence the same samples, opacities and termination);
//   2. run the deferred MLP forward and backward in FP32: dL/dC_d = dL/dC + (dh/dC_d)^T dL/dC,
//      dL/dF = (dh/dF)^T dL/dC, and the weight gradients, summed over the warp's pixels as small
//      matrix products in shared memory and accumulated per CTA;
//   3. march again front to back, recomputing transmittance instead of storing per-sample
//      state.  With G = (dL/dC_d, dL/dF), v_i = (c_i, f_i) and A_i = sum_{j<=i} w_j G.v_j, the
//      gradient of Eq. 1 / Eq. 2 with respect to a sample's opacity is
//          dL/dalpha_i = T_i G.v_i - S_i / (1 - alpha_i),   S_i = G.C - A_i,
//      because S_i, the contribution of the samples behind i, carries a factor (1 - alpha_i).
//      Through alpha = 1 - exp(-tau delta) and tau = exp(t~_0) the factor cancels:
//          dL/dt~_0 = (T_i G.v_i (1 - alpha_i) - S_i) tau delta,
//      so nothing is divided by a vanishing 1 - alpha.  With the two sigmoids this gives dL/dt~
//      (8 channels), scattered into the grid and plane gradients with the interpolation weights
//      (float4 atomics).
#pragma once

#include <type_traits>

#include "render.cuh"

namespace merf {

struct BackwardParams {
    FieldView fv;
    OccView occ;
    const float *mlp;
    const float *d_out;     // [n][H][W][3] dL/dC
    const float *aux;       // forward's [n][H][W][kAuxSize] (C_d, F, ...) or null: march again
    float *g_grid;          // [L][L][L][8]
    float *g_planes;        // [3][R][R][8]
    float *g_mlp;           // [883]
    int W, H, cam0;
    float step, t_term;
    int early_term;
    CamBlock cams;
};

// Add w g at texel `key` of `base` (8 floats per texel; key < 0: nothing), merging with the
// horizontally adjacent pixel (lane ^ 1) when both add to the same texel: the even lane adds the
// pair's sum and the odd lane skips its atomics.  m: the lanes executing this call together.
// Key: int when every texel index fits (the 32-bit variant), else long long.  The float offset
// key * 8 is formed in 64 bits, so it cannot wrap whatever the key's type.
template <typename Key>
__device__ __forceinline__ void atomic_add8_pair(float *base, Key key, const float g[8], float w, unsigned m)
{
    const int lane = threadIdx.x & 31;
    const Key pk = __shfl_xor_sync(m, key, 1);
    const bool merge = key >= 0 && pk == key && ((m >> (lane ^ 1)) & 1u);
    float v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = w * g[c];
    if (__any_sync(m, merge)) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float o = __shfl_xor_sync(m, v[c], 1);
            if (merge) v[c] += o;
        }
    }
    if (key < 0 || (merge && (lane & 1))) return;
    float *dst = base + (long long)key * 8;
    atomicAdd(reinterpret_cast<float4 *>(dst), make_float4(v[0], v[1], v[2], v[3]));
    atomicAdd(reinterpret_cast<float4 *>(dst + 4), make_float4(v[4], v[5], v[6], v[7]));
}

// Add g (per channel) times the interpolation weights of p to the dense grid and plane gradients.
template <int kGeo>
__device__ __forceinline__ void scatter_f32(const FieldView &fv, float *g_grid, float *g_planes, float p0, float p1,
                                            float p2, const float g[8])
{
    using Idx = typename GatherIndex<kGeo>::T;
    using Key = typename std::conditional<sizeof(Idx) == 4, int, long long>::type;   // signed: -1 = none
    const float sL = (float)fv.L * 0.25f;
    const int hL = fv.L >> 1, L = fv.L;
    int x0, y0, z0;
    float fx, fy, fz;
    texel_coord(p0, sL, hL, L, x0, fx);
    texel_coord(p1, sL, hL, L, y0, fy);
    texel_coord(p2, sL, hL, L, z0, fz);
    const unsigned m = __activemask();
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
        const float w = (cx ? fx : 1.0f - fx) * (cy ? fy : 1.0f - fy) * (cz ? fz : 1.0f - fz);
        const Idx gi = ((Idx)(z0 + cz) * L + (y0 + cy)) * L + (x0 + cx);
        const bool ok = w != 0.0f && MERF_IN_RANGE(gi, (long long)L * L * L, kBadDense);
        atomic_add8_pair<Key>(g_grid, ok ? (Key)gi : (Key)-1, g, w, m);
    }
    const float sR = (float)fv.R * 0.25f;
    const int hR = fv.R >> 1, R = fv.R;
    int u0[3];
    float fu[3];
    texel_coord(p0, sR, hR, R, u0[0], fu[0]);
    texel_coord(p1, sR, hR, R, u0[1], fu[1]);
    texel_coord(p2, sR, hR, R, u0[2], fu[2]);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int ca = q == 0 ? 1 : 0, ra = q == 2 ? 1 : 2;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int cu = c & 1, cv = c >> 1;
            const float w = (cu ? fu[ca] : 1.0f - fu[ca]) * (cv ? fu[ra] : 1.0f - fu[ra]);
            const Idx pi = ((Idx)q * R + u0[ra] + cv) * R + u0[ca] + cu;
            const bool ok = w != 0.0f && MERF_IN_RANGE(pi, 3LL * R * R, kBadDense);
            atomic_add8_pair<Key>(g_planes, ok ? (Key)pi : (Key)-1, g, w, m);
        }
    }
}

// Deferred MLP forward + backward for one pixel (FP32), without the weight gradients: from
// dL/dh = gh it returns x (the 34 inputs), a1, a2 (the ReLU activations), dz1, dz2 (gradients of
// the two pre-activations) and dL/dx for x[0..6] = (C_d, F).
__device__ __forceinline__ void mlp_backward_f32(const float *w, const float cd[3], const float f[4], const float d[3],
                                                 const float gh[3], float x[34], float a1[16], float a2[16],
                                                 float dz1[16], float dz2[16], float gx7[7])
{
    x[0] = cd[0]; x[1] = cd[1]; x[2] = cd[2];
    x[3] = f[0]; x[4] = f[1]; x[5] = f[2]; x[6] = f[3];
    x[7] = d[0]; x[8] = d[1]; x[9] = d[2];
    posenc(d, x);          // the forward's encoding, bit for bit
    const float *W0 = w, *b0 = w + 544, *W1 = w + 560, *b1 = w + 816, *W2 = w + 832;
#pragma unroll
    for (int o = 0; o < 16; ++o) a1[o] = b0[o];
#pragma unroll
    for (int i = 0; i < 34; ++i)
#pragma unroll
        for (int o = 0; o < 16; ++o) a1[o] = fmaf(x[i], W0[i * 16 + o], a1[o]);
#pragma unroll
    for (int o = 0; o < 16; ++o) a1[o] = fmaxf(a1[o], 0.0f);
#pragma unroll
    for (int o = 0; o < 16; ++o) a2[o] = b1[o];
#pragma unroll
    for (int i = 0; i < 16; ++i)
#pragma unroll
        for (int o = 0; o < 16; ++o) a2[o] = fmaf(a1[i], W1[i * 16 + o], a2[o]);
    // ReLU derivative from the activations: a > 0 exactly where the pre-activation is
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        a2[i] = fmaxf(a2[i], 0.0f);
        float acc = 0.0f;
#pragma unroll
        for (int o = 0; o < 3; ++o) acc = fmaf(W2[i * 3 + o], gh[o], acc);
        dz2[i] = a2[i] > 0.0f ? acc : 0.0f;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        float acc = 0.0f;
#pragma unroll
        for (int o = 0; o < 16; ++o) acc = fmaf(W1[i * 16 + o], dz2[o], acc);
        dz1[i] = a1[i] > 0.0f ? acc : 0.0f;
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        float acc = 0.0f;
#pragma unroll
        for (int o = 0; o < 16; ++o) acc = fmaf(W0[i * 16 + o], dz1[o], acc);
        gx7[i] = acc;
    }
}

// Per-warp staging of the 32 pixels' MLP vectors for the weight gradients (rows padded to odd
// strides, so that the 32 lanes writing their own rows hit 32 different banks).
constexpr int kXs = 35, kVs = 17;
constexpr int kStageFloats = 32 * kXs + 32 * kVs;      // phase 1: x and dz1; later phases reuse it

// Weight gradients of the warp's 32 pixels, added into the CTA's accumulator gw (all 32 lanes
// call; lanes without a pixel pass gh = 0, hence zero dz1, dz2).  Each parameter's gradient is a
// sum over the pixels of an outer-product term, e.g. dL/dW0[i][o] = sum_p x_p[i] dz1_p[o]: the
// vectors go through shared memory and lane l sums the column o = l mod 16 for the rows of its
// parity, so each lane adds 17 + 8 + 2 distinct entries (plus biases) with no lane conflicts.
__device__ __forceinline__ void mlp_weight_grads_warp(float *gw, float *st, const float x[34], const float a1[16],
                                                      const float a2[16], const float dz1[16], const float dz2[16],
                                                      const float gh[3])
{
    const int lane = threadIdx.x & 31, o = lane & 15, r0 = lane >> 4;
    float *xs = st, *vs = st + 32 * kXs;
    // W0 [34][16] and b0
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 34; ++i) xs[lane * kXs + i] = x[i];
#pragma unroll
    for (int i = 0; i < 16; ++i) vs[lane * kVs + i] = dz1[i];
    __syncwarp();
    {
        float acc[17], bsum = 0.0f;
#pragma unroll
        for (int m = 0; m < 17; ++m) acc[m] = 0.0f;
#pragma unroll 2
        for (int p = 0; p < 32; ++p) {
            const float d = vs[p * kVs + o];
            bsum += d;
#pragma unroll
            for (int m = 0; m < 17; ++m) acc[m] = fmaf(xs[p * kXs + r0 + 2 * m], d, acc[m]);
        }
#pragma unroll
        for (int m = 0; m < 17; ++m)
            if (acc[m] != 0.0f) atomicAdd(gw + (r0 + 2 * m) * 16 + o, acc[m]);
        if (r0 == 0 && bsum != 0.0f) atomicAdd(gw + 544 + o, bsum);
    }
    // W1 [16][16] and b1
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 16; ++i) xs[lane * kVs + i] = a1[i];
#pragma unroll
    for (int i = 0; i < 16; ++i) vs[lane * kVs + i] = dz2[i];
    __syncwarp();
    {
        float acc[8], bsum = 0.0f;
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[m] = 0.0f;
#pragma unroll 2
        for (int p = 0; p < 32; ++p) {
            const float d = vs[p * kVs + o];
            bsum += d;
#pragma unroll
            for (int m = 0; m < 8; ++m) acc[m] = fmaf(xs[p * kVs + r0 + 2 * m], d, acc[m]);
        }
#pragma unroll
        for (int m = 0; m < 8; ++m)
            if (acc[m] != 0.0f) atomicAdd(gw + 560 + (r0 + 2 * m) * 16 + o, acc[m]);
        if (r0 == 0 && bsum != 0.0f) atomicAdd(gw + 816 + o, bsum);
    }
    // W2 [16][3] and b2
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 16; ++i) xs[lane * kVs + i] = a2[i];
#pragma unroll
    for (int k = 0; k < 3; ++k) vs[lane * kVs + k] = gh[k];
    __syncwarp();
    {
        float acc[2] = {0.0f, 0.0f}, bsum = 0.0f;
        const int e1 = lane + 32;                  // entries lane and lane + 32 of the 48
#pragma unroll 2
        for (int p = 0; p < 32; ++p) {
            acc[0] = fmaf(xs[p * kVs + lane / 3], vs[p * kVs + lane % 3], acc[0]);
            if (e1 < 48) acc[1] = fmaf(xs[p * kVs + e1 / 3], vs[p * kVs + e1 % 3], acc[1]);
            if (lane < 3) bsum += vs[p * kVs + lane];
        }
        if (acc[0] != 0.0f) atomicAdd(gw + 832 + lane, acc[0]);
        if (e1 < 48 && acc[1] != 0.0f) atomicAdd(gw + 832 + e1, acc[1]);
        if (lane < 3 && bsum != 0.0f) atomicAdd(gw + 880 + lane, bsum);
    }
    __syncwarp();
}

// kGeo: kGeoDense32 (32-bit offsets) or kGeoRuntime (64-bit), as the host chose for the scene.
template <int kGeo>
__global__ void __launch_bounds__(kThreads, 4) backward_kernel(const __grid_constant__ BackwardParams P)
{
    __shared__ float wsm[kMlpParams];
    __shared__ float gsm[kMlpParams];
    __shared__ float stage[kThreads / 32][kStageFloats];
    for (int t = threadIdx.x; t < kMlpParams; t += kThreads) {
        wsm[t] = __ldg(P.mlp + t);
        gsm[t] = 0.0f;
    }
    __syncthreads();
    int i, j;
    pixel_of_thread(i, j);
    const int cl = blockIdx.z;
    const bool live = i < P.W && j < P.H;
    const size_t pix = live ? ((size_t)(P.cam0 + cl) * P.H + j) * P.W + i : 0;
    const float *cam = P.cams.m[cl];
    float gC[3] = {0.0f, 0.0f, 0.0f};
    RayState r;
    ray_state_init(r);
    if (live) {
        gC[0] = P.d_out[pix * 3 + 0];
        gC[1] = P.d_out[pix * 3 + 1];
        gC[2] = P.d_out[pix * 3 + 2];
        if (P.aux) {   // C_d and F as the forward pass composited them
            const float *a = P.aux + pix * kAuxSize;
            r.cd[0] = a[0]; r.cd[1] = a[1]; r.cd[2] = a[2];
            r.F[0] = a[3]; r.F[1] = a[4]; r.F[2] = a[5]; r.F[3] = a[6];
            float o[3];
            ray_f32(cam, i, j, o, r.d);
        } else {
            march_ray<1, 0, kGeo>(P.fv, P.occ, cam, i, j, P.step, P.t_term, P.early_term, r);
        }
    }
    // the whole warp: MLP backward per lane, weight gradients reduced across the warp
    float gx7[7];
    {
        float x[34], a1[16], a2[16], dz1[16], dz2[16];
        mlp_backward_f32(wsm, r.cd, r.F, r.d, gC, x, a1, a2, dz1, dz2, gx7);
        mlp_weight_grads_warp(gsm, stage[threadIdx.x >> 5], x, a1, a2, dz1, dz2, gC);
    }
    if (live) {
        const float Gc[3] = {gC[0] + gx7[0], gC[1] + gx7[1], gC[2] + gx7[2]};
        const float Gf[4] = {gx7[3], gx7[4], gx7[5], gx7[6]};
        const float Gtot = Gc[0] * r.cd[0] + Gc[1] * r.cd[1] + Gc[2] * r.cd[2] + Gf[0] * r.F[0] + Gf[1] * r.F[1] +
                           Gf[2] * r.F[2] + Gf[3] * r.F[3];
        const float Gabs = fabsf(Gc[0]) + fabsf(Gc[1]) + fabsf(Gc[2]) + fabsf(Gf[0]) + fabsf(Gf[1]) + fabsf(Gf[2]) +
                           fabsf(Gf[3]);
        // second march, front to back, recomputing T
        float o[3], d[3];
        ray_f32(cam, i, j, o, d);
        Walker wk;
        wk.init(o, d, P.step);
        float T = 1.0f, A = 0.0f;
        for (;;) {
            float p0, p1, p2;
            if (!wk.next_sample<typename GatherIndex<kGeo>::T>(P.occ, p0, p1, p2)) break;
            float t8[8];
            field_f32<kGeo>(P.fv, p0, p1, p2, t8);
            const float tau = __expf(t8[0]);
            const float dw = wk.delta_world(wk.k);
            const float alpha = 1.0f - __expf(-tau * dw);
            if (alpha > 0.0f) {
                float c[3], f[4];
#pragma unroll
                for (int k = 0; k < 3; ++k) c[k] = sigmoid_f(t8[1 + k]);
#pragma unroll
                for (int k = 0; k < 4; ++k) f[k] = sigmoid_f(t8[4 + k]);
                const float w = alpha * T;
                const float Gv = Gc[0] * c[0] + Gc[1] * c[1] + Gc[2] * c[2] + Gf[0] * f[0] + Gf[1] * f[1] +
                                 Gf[2] * f[2] + Gf[3] * f[3];
                A = fmaf(w, Gv, A);
                const float om = 1.0f - alpha;
                // dL/dt~_0 = dL/dalpha (1 - alpha) tau delta = (T G.v (1 - alpha) - S) tau delta with
                // S = G.C - A the contribution behind the sample: no division by 1 - alpha.  S is
                // clamped to its bound |S| <= T (1 - alpha) sum |G|, which removes the rounding noise
                // of the subtraction where almost nothing lies behind.
                const float sbound = T * om * Gabs;
                const float S = fminf(fmaxf(Gtot - A, -sbound), sbound);
                float g[8];
                g[0] = (T * Gv * om - S) * (tau * dw);
#pragma unroll
                for (int k = 0; k < 3; ++k) g[1 + k] = w * Gc[k] * c[k] * (1.0f - c[k]);
#pragma unroll
                for (int k = 0; k < 4; ++k) g[4 + k] = w * Gf[k] * f[k] * (1.0f - f[k]);
                scatter_f32<kGeo>(P.fv, P.g_grid, P.g_planes, p0, p1, p2, g);
                T = T * om;
                if (P.early_term && T < P.t_term) break;
            }
            ++wk.k;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kMlpParams; t += kThreads)
        if (gsm[t] != 0.0f) atomicAdd(P.g_mlp + t, gsm[t]);
}

}  // namespace merf
