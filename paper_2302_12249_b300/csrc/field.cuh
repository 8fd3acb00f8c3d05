// field.cuh -- the MERF feature field at a contracted point (Sec. 3.1, Sec. 4.2) for sm_103a.
//
// t~(p) = V(x, y, z) + P_x(y, z) + P_y(x, z) + P_z(x, y): trilinear interpolation in the
// low-resolution 3D grid plus bilinear interpolation in three high-resolution planes, each
// texel dequantised as 2 m k / 255 - m (m = 14 for density, 7 otherwise).  Because the
// dequantisation is affine and interpolation weights sum to one, the kernel interpolates raw
// byte values and dequantises the sum once per channel:
//     t~_c = (2 m_c / 255) * sum_w w k_c  -  m_c * (W_V + 3),
// with W_V the weight of the 3D-grid corners that are stored (a voxel of a block that is not
// stored contributes nothing).
//
// Layout in HBM: every texel is 8 bytes (one uint2: channels 0..3 in .x, 4..7 in .y), so
// one 64-bit load fetches density and appearance of a corner.  The 3D grid is block-sparse:
// an int32 index grid over (L/B)^3 blocks points into an atlas of B^3-voxel blocks laid out
// [z][y][x].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace merf {

struct FieldView {
    const int32_t *index_grid;   // [(L/B)^3]
    const uint2 *atlas;          // [n_blocks][B][B][B]
    const uint2 *planes;         // [3][R][R]
    const float4 *grid_f32;      // dense storage: [L][L][L][2]
    const float4 *planes_f32;    // dense storage: [3][R][R][2]
    int L, B, log2B, nb, R;
};

// Continuous texel index u = (p + 2) N / 4 - 1/2 split into an integer part and a fraction
// without rounding: p * N/4 is exact when N/4 is a power of two, floor and the difference are
// exact, and the +-1/2 shift of the remainder is exact or below one float ulp of 1/2.
__device__ __forceinline__ void texel_coord(float p, float scale, int half, int N, int &i0, int &i1,
                                            float &f)
{
    const float a = __fmul_rn(p, scale);
    const float fl = floorf(a);
    const float r = a - fl;
    const int ib = (int)fl + half;
    if (r >= 0.5f) { i0 = ib; f = r - 0.5f; } else { i0 = ib - 1; f = r + 0.5f; }
    i1 = min(max(i0 + 1, 0), N - 1);
    i0 = min(max(i0, 0), N - 1);
}

__device__ __forceinline__ float byte_of(uint32_t w, int b)
{
    return (float)((w >> (8 * b)) & 0xffu);
}

// The 20 texels of one sample: 8 grid corners and 4 texels in each plane, with weights.
struct Taps {
    uint2 v[20];
    float w[20];
};

__device__ __forceinline__ void gather_u8(const FieldView &fv, float p0, float p1, float p2, Taps &t)
{
    const float sL = (float)fv.L * 0.25f;
    const int hL = fv.L >> 1;
    int x0, x1, y0, y1, z0, z1;
    float fx, fy, fz;
    texel_coord(p0, sL, hL, fv.L, x0, x1, fx);
    texel_coord(p1, sL, hL, fv.L, y0, y1, fy);
    texel_coord(p2, sL, hL, fv.L, z0, z1, fz);
    const int sh = fv.log2B, msk = fv.B - 1, nb = fv.nb, B = fv.B;
    const int bx0 = x0 >> sh, bx1 = x1 >> sh, by0 = y0 >> sh, by1 = y1 >> sh, bz0 = z0 >> sh, bz1 = z1 >> sh;
    const int b000 = __ldg(fv.index_grid + (bz0 * nb + by0) * nb + bx0);
    const bool one = (bx0 == bx1) & (by0 == by1) & (bz0 == bz1);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
        const int bx = cx ? bx1 : bx0, by = cy ? by1 : by0, bz = cz ? bz1 : bz0;
        const int blk = (one || c == 0) ? b000 : __ldg(fv.index_grid + (bz * nb + by) * nb + bx);
        const int lx = (cx ? x1 : x0) & msk, ly = (cy ? y1 : y0) & msk, lz = (cz ? z1 : z0) & msk;
        const float w = (cx ? fx : 1.0f - fx) * (cy ? fy : 1.0f - fy) * (cz ? fz : 1.0f - fz);
        if (blk >= 0) {
            t.v[c] = __ldg(fv.atlas + (((size_t)blk * B + lz) * B + ly) * B + lx);
            t.w[c] = w;
        } else {
            t.v[c] = make_uint2(0u, 0u);
            t.w[c] = 0.0f;
        }
    }
    const float sR = (float)fv.R * 0.25f;
    const int hR = fv.R >> 1, R = fv.R;
    int u0[3], u1[3];
    float fu[3];
    texel_coord(p0, sR, hR, R, u0[0], u1[0], fu[0]);
    texel_coord(p1, sR, hR, R, u0[1], u1[1], fu[1]);
    texel_coord(p2, sR, hR, R, u0[2], u1[2], fu[2]);
    // plane q: columns along axis (1, 0, 0)[q], rows along axis (2, 2, 1)[q]
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int ca = q == 0 ? 1 : 0, ra = q == 2 ? 1 : 2;
        const uint2 *base = fv.planes + (size_t)q * R * R;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int cu = c & 1, cv = c >> 1;
            const int col = cu ? u1[ca] : u0[ca], row = cv ? u1[ra] : u0[ra];
            t.v[8 + 4 * q + c] = __ldg(base + (size_t)row * R + col);
            t.w[8 + 4 * q + c] = (cu ? fu[ca] : 1.0f - fu[ca]) * (cv ? fu[ra] : 1.0f - fu[ra]);
        }
    }
}

// Density pre-activation t~_0 from gathered taps.
__device__ __forceinline__ float density_u8(const Taps &t)
{
    float k = 0.0f, wv = 0.0f;
#pragma unroll
    for (int i = 0; i < 20; ++i) k = fmaf(t.w[i], byte_of(t.v[i].x, 0), k);
#pragma unroll
    for (int i = 0; i < 8; ++i) wv += t.w[i];
    return k * (28.0f / 255.0f) - 14.0f * (wv + 3.0f);
}

// Appearance pre-activations t~_1..7.
__device__ __forceinline__ void appearance_u8(const Taps &t, float out[7])
{
    float wv = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) wv += t.w[i];
    const float off = 7.0f * (wv + 3.0f);
#pragma unroll
    for (int c = 1; c < 8; ++c) {
        float k = 0.0f;
#pragma unroll
        for (int i = 0; i < 20; ++i) k = fmaf(t.w[i], byte_of(c < 4 ? t.v[i].x : t.v[i].y, c & 3), k);
        out[c - 1] = k * (14.0f / 255.0f) - off;
    }
}

// Dense float storage: all eight channels of all 20 taps, summed.
__device__ __forceinline__ void field_f32(const FieldView &fv, float p0, float p1, float p2, float out[8])
{
    const float sL = (float)fv.L * 0.25f;
    const int hL = fv.L >> 1, L = fv.L;
    int x[2], y[2], z[2];
    float fx, fy, fz;
    texel_coord(p0, sL, hL, L, x[0], x[1], fx);
    texel_coord(p1, sL, hL, L, y[0], y[1], fy);
    texel_coord(p2, sL, hL, L, z[0], z[1], fz);
#pragma unroll
    for (int c = 0; c < 8; ++c) out[c] = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
        const float w = (cx ? fx : 1.0f - fx) * (cy ? fy : 1.0f - fy) * (cz ? fz : 1.0f - fz);
        const float4 *q = fv.grid_f32 + (((size_t)z[cz] * L + y[cy]) * L + x[cx]) * 2;
        const float4 a = __ldg(q), b = __ldg(q + 1);
        out[0] = fmaf(w, a.x, out[0]); out[1] = fmaf(w, a.y, out[1]);
        out[2] = fmaf(w, a.z, out[2]); out[3] = fmaf(w, a.w, out[3]);
        out[4] = fmaf(w, b.x, out[4]); out[5] = fmaf(w, b.y, out[5]);
        out[6] = fmaf(w, b.z, out[6]); out[7] = fmaf(w, b.w, out[7]);
    }
    const float sR = (float)fv.R * 0.25f;
    const int hR = fv.R >> 1, R = fv.R;
    int u0[3], u1[3];
    float fu[3];
    texel_coord(p0, sR, hR, R, u0[0], u1[0], fu[0]);
    texel_coord(p1, sR, hR, R, u0[1], u1[1], fu[1]);
    texel_coord(p2, sR, hR, R, u0[2], u1[2], fu[2]);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int ca = q == 0 ? 1 : 0, ra = q == 2 ? 1 : 2;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int cu = c & 1, cv = c >> 1;
            const int col = cu ? u1[ca] : u0[ca], row = cv ? u1[ra] : u0[ra];
            const float w = (cu ? fu[ca] : 1.0f - fu[ca]) * (cv ? fu[ra] : 1.0f - fu[ra]);
            const float4 *t = fv.planes_f32 + (((size_t)q * R + row) * R + col) * 2;
            const float4 a = __ldg(t), b = __ldg(t + 1);
            out[0] = fmaf(w, a.x, out[0]); out[1] = fmaf(w, a.y, out[1]);
            out[2] = fmaf(w, a.z, out[2]); out[3] = fmaf(w, a.w, out[3]);
            out[4] = fmaf(w, b.x, out[4]); out[5] = fmaf(w, b.y, out[5]);
            out[6] = fmaf(w, b.z, out[6]); out[7] = fmaf(w, b.w, out[7]);
        }
    }
}

}  // namespace merf
