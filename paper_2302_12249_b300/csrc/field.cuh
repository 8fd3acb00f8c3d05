// field.cuh -- the MERF feature field at a contracted point (Sec. 3.1, Sec. 4.2) for sm_103a.
//
// t~(p) = V(x, y, z) + P_x(y, z) + P_y(x, z) + P_z(x, y): trilinear interpolation in the
// low-resolution 3D grid plus bilinear interpolation in three high-resolution planes, each
// texel dequantised as 2 m k / 255 - m (m = 14 for density, 7 otherwise).  Because the
// dequantisation is affine and interpolation weights sum to one, the kernel interpolates raw
// byte values (exactly, in integers: dot_sums below) and dequantises the sum once per channel:
//     t~_c = (2 m_c / 255) * sum_w w k_c  -  m_c * (W_V + 3),
// with W_V the weight of the 3D-grid corners that are stored (a voxel of a block that is not
// stored contributes nothing).  A grid-only scene (no planes, R = 0: the SNeRG++-style baseline
// of Sec. 6) has t~ = V and the offset m_c W_V.
//
// Layout in HBM.  A texel is 8 bytes (channels 0..7), and every texel is stored together with
// its +x neighbour (the +u neighbour in a plane) as one 16-byte texel pair, the two texels' bytes
// interleaved (a0, b0, a1, b1, ..., a7, b7): one 128-bit load fetches density and appearance of
// two corners in the byte order the interpolation's dot products take, so no byte permute is
// left per sample (the pair of a row's last texel has a zero upper texel).  This doubles the
// texel storage against 8 bytes per texel, for 10 loads and 40 permutes fewer per sample.  The
// 3D grid is block-sparse: an int32 index grid over (L/B)^3 blocks holds, for a stored block,
// its atlas slot in bits 0..23 and in bits 24..30 a mask of which of its +x/+y/+z neighbour
// blocks are not stored (neighbour dx + 2 dy + 4 dz in 1..7 at bit 23 + that number); -1 marks
// a block that is not stored.  Each atlas slot holds (B+1)^3 voxel pairs [z][y][x]: the block
// plus a one-voxel apron copied from its +x/+y/+z neighbours, so the four corner pairs of any
// sample whose lowest corner lies in the block are one base address plus constant offsets.
// For the 3D grid, clamp-to-edge is folded into the integer coordinate and weight (lowest corner
// kept in [0, N-2]), so no lookup leaves the array.  The planes are stored [3][R+2][R+2] (texel
// pairs) with a one-texel border that repeats their edge texels, so their taps need no clamp.
// The occupancy grids are not read here (the traversal tests them before a sample is evaluated).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "debug.cuh"
#include "geometry.h"

namespace merf {

struct FieldView {
    const int32_t *index_grid;   // [(L/B)^3] slot | missing-neighbour mask << 24, or -1
    const uint4 *atlas;          // [n_blocks][B+1][B+1][B+1] texel pairs (x, x + 1)
    const uint4 *planes;         // [3][R+2][R+2] texel pairs (u, u + 1): one-texel clamp-to-edge border
    const float4 *grid_f32;      // dense storage: [L][L][L][2]
    const float4 *planes_f32;    // dense storage: [3][R][R][2]
    int L, B, log2B, nb, R;
    int n_blocks;                // stored blocks (atlas slots)
};

// Lowest corner i0 and weight f of the upper corner for the continuous texel index
// u = (p + 2) N / 4 - 1/2 with clamp-to-edge.  a = p N/4 is exact when N/4 is a power of two;
// adding 1.5 * 2^23 rounds it to the nearest integer n (held in the low mantissa bits, |a| <
// 2^22), which is read back exactly; d = a - n in [-1/2, 1/2] is exact, so
// u = (n - 1 + N/2) + (d + 1/2) with d + 1/2 in [0, 1] rounded at most once, below 2^-25.
// Outside [0, N-1] the clamped value is expressed as i0 in {0, N-2} with f in {0, 1}.
__device__ __forceinline__ void texel_coord(float p, float scale, int half, int N, int &i0, float &f)
{
    const float a = __fmul_rn(p, scale);
    const float t = __fadd_rn(a, 12582912.0f);
    const float n = __fsub_rn(t, 12582912.0f);
    i0 = (int)(__float_as_uint(t) - 0x4B400000u) - 1 + half;
    f = __fadd_rn(__fsub_rn(a, n), 0.5f);
    if (i0 < 0) { i0 = 0; f = 0.0f; }
    if (i0 > N - 2) { i0 = N - 2; f = 1.0f; }
}

// The same for a plane stored with a one-texel border that repeats its edge texels: the lowest
// tap in bordered coordinates is i0 + 1 = n + N/2 in [0, N], with f unchanged.  Clamp-to-edge
// then needs no clamp (a tap on the border reads the edge value), because every contracted
// point lies in [-2, 2]; the index is still bounded to [0, N] so that no tap leaves the array.
__device__ __forceinline__ void plane_coord(float p, float scale, int half, int N, int &i0, float &f)
{
    const float a = __fmul_rn(p, scale);
    const float t = __fadd_rn(a, 12582912.0f);
    const float n = __fsub_rn(t, 12582912.0f);
    i0 = min(max((int)(__float_as_uint(t) - 0x4B400000u) + half, 0), N);
    f = __fadd_rn(__fsub_rn(a, n), 0.5f);
}

// The 20 texels of one sample (8 grid corners, 4 texels in each plane) as 10 texel pairs, each
// pair's bytes interleaved (pair_bytes), and their weights.
struct Taps {
    uint4 q[10];
    float fx, fy, fz;       // grid fractions
    float fu[3];            // plane fractions along x, y, z
    float wv;               // weight of the stored grid corners
};

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    // PTX prmt, default mode: a selector nibble with its high bit set replicates the selected
    // byte's sign bit over the output byte (used here on bytes whose top bit is zero, for zeros)
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// The byte pairs of texels a and b: channels (0, 1), (2, 3), (4, 5), (6, 7), each as
// (a.c, b.c, a.c', b.c'): the two texels' bytes interleaved, as the scene stores its texel pairs.
__device__ __forceinline__ uint4 pair_bytes(uint2 a, uint2 b)
{
    return make_uint4(prmt(a.x, b.x, 0x5140u), prmt(a.x, b.x, 0x7362u), prmt(a.y, b.y, 0x5140u),
                      prmt(a.y, b.y, 0x7362u));
}

// The lower texel of an interleaved pair (its even bytes).
__device__ __forceinline__ uint2 pair_lower(uint4 q)
{
    return make_uint2(prmt(q.x, q.y, 0x6420u), prmt(q.z, q.w, 0x6420u));
}

// Trilinear weight of grid corner c.  A corner that is not stored holds zero bytes (the apron
// of a missing neighbour is zero-filled and the slow path loads zeros), so it contributes
// nothing to any weighted byte sum without masking; only W_V excludes it.
__device__ __forceinline__ float grid_w(const Taps &t, int c)
{
    return ((c & 1) ? t.fx : 1.0f - t.fx) * ((c & 2) ? t.fy : 1.0f - t.fy) * ((c & 4) ? t.fz : 1.0f - t.fz);
}

// W_V: the sum of the weights of the stored corners (bit c of mask set: corner c stored).
__device__ __forceinline__ float stored_weight(const Taps &t, uint32_t mask)
{
    float wv = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) wv += ((mask >> c) & 1u) ? grid_w(t, c) : 0.0f;
    return wv;
}

// Lowest corner in a block that is not stored: every corner is looked up on its own (as the
// lower texel of its stored pair) and the pairs are interleaved here.
__device__ __forceinline__ void gather_grid_slow(const FieldView &fv, int x0, int y0, int z0, Taps &t)
{
    const int sh = fv.log2B, msk = fv.B - 1, nb = fv.nb, B1 = fv.B + 1;
    uint32_t gmask = 0u;
    uint2 v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int x = x0 + (c & 1), y = y0 + ((c >> 1) & 1), z = z0 + (c >> 2);
        const int gi = ((z >> sh) * nb + (y >> sh)) * nb + (x >> sh);
        const int ent = MERF_IN_RANGE(gi, nb * nb * nb, kBadIndexGrid) ? __ldg(fv.index_grid + gi) : -1;
        const size_t slot = (size_t)(ent & 0xffffff);
        const size_t ai = ((slot * B1 + (z & msk)) * B1 + (y & msk)) * B1 + (x & msk);
        if (ent >= 0 && MERF_IN_RANGE(ai, (long long)fv.n_blocks * B1 * B1 * B1, kBadAtlas)) {
            v[c] = pair_lower(__ldg(fv.atlas + ai));
            gmask |= 1u << c;
        } else {
            v[c] = make_uint2(0u, 0u);
        }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) t.q[p] = pair_bytes(v[2 * p], v[2 * p + 1]);
    t.wv = stored_weight(t, gmask);
}

// The gather variants (kGeoRuntime, kGeoPaper, kGeoGridOnly, kGeoGridOnlyWide, kGeoDense32) and the host's choice among them are
// in geometry.h.
template <int kGeo>
constexpr int kPlaneSources = kGridOnly<kGeo> ? 0 : 3;          // planes that add to the grid
template <int kGeo>
constexpr int kTaps = 8 + 4 * kPlaneSources<kGeo>;               // texels per sample
// Offset type of the gather and occupancy indices: 32-bit for the variants the host picks only when
// offsets_fit_32 holds (kGeoPaper, kGeoGridOnly) or dense_offsets_fit_32 (kGeoDense32), 64-bit for
// the others.
template <int kGeo>
struct GatherIndex { using T = size_t; };
template <>
struct GatherIndex<kGeoPaper> { using T = uint32_t; };
template <>
struct GatherIndex<kGeoGridOnly> { using T = uint32_t; };
template <>
struct GatherIndex<kGeoDense32> { using T = uint32_t; };

template <int kGeo>
__device__ __forceinline__ void gather_u8(const FieldView &fv, float p0, float p1, float p2, Taps &t)
{
    using Idx = typename GatherIndex<kGeo>::T;
    const int L = kGeo == kGeoPaper ? 512 : fv.L;
    const int sh = kGeo == kGeoPaper ? 4 : fv.log2B;
    const int nb = kGeo == kGeoPaper ? 32 : fv.nb;
    const int Rg = kGeo == kGeoPaper ? 2048 : fv.R;
    const float sL = (float)L * 0.25f;
    const int hL = L >> 1;
    int x0, y0, z0;
    texel_coord(p0, sL, hL, L, x0, t.fx);
    texel_coord(p1, sL, hL, L, y0, t.fy);
    texel_coord(p2, sL, hL, L, z0, t.fz);
    const int msk = (1 << sh) - 1, B1 = (1 << sh) + 1;
    const int gi = ((z0 >> sh) * nb + (y0 >> sh)) * nb + (x0 >> sh);
    const int ent = MERF_IN_RANGE(gi, nb * nb * nb, kBadIndexGrid) ? __ldg(fv.index_grid + gi) : -1;
    if (ent >= 0) {
        const int lx = x0 & msk, ly = y0 & msk, lz = z0 & msk;
        const Idx ai = ((Idx)(ent & 0xffffff) * B1 + lz) * B1 * B1 + ly * B1 + lx;
        // bounds-checked build: the farthest corner is ai + B1^2 + B1 + 1
        if (!MERF_IN_RANGE(ai + B1 * B1 + B1 + 1, (long long)fv.n_blocks * B1 * B1 * B1, kBadAtlas)) {
#pragma unroll
            for (int c = 0; c < 4; ++c) t.q[c] = make_uint4(0u, 0u, 0u, 0u);
            t.wv = 0.0f;
            goto grid_done;
        }
        const uint4 *base = fv.atlas + ai;
        const int sy = B1, sz = B1 * B1;
        t.q[0] = __ldg(base);
        t.q[1] = __ldg(base + sy);
        t.q[2] = __ldg(base + sz);
        t.q[3] = __ldg(base + sz + sy);
        t.wv = 1.0f;
        const uint32_t miss = ((uint32_t)ent >> 24) << 1;     // bit n: neighbour n not stored
        if (miss) {
            uint32_t gmask = 0xffu;
            // corners that fall in the apron of a neighbour that is not stored
            const int ex = lx == msk, ey = ly == msk, ez = lz == msk;
#pragma unroll
            for (int c = 1; c < 8; ++c) {
                const int nbr = ((c & 1) & ex) | ((((c >> 1) & 1) & ey) << 1) | ((((c >> 2) & 1) & ez) << 2);
                if ((miss >> nbr) & 1u) gmask &= ~(1u << c);
            }
            t.wv = stored_weight(t, gmask);
        }
    } else {
        gather_grid_slow(fv, x0, y0, z0, t);
    }
grid_done:;
    if constexpr (kGridOnly<kGeo>) return;
    const float sR = (float)Rg * 0.25f;
    const int hR = Rg >> 1, R = Rg, Rp = Rg + 2;
    int u0[3];
    plane_coord(p0, sR, hR, R, u0[0], t.fu[0]);
    plane_coord(p1, sR, hR, R, u0[1], t.fu[1]);
    plane_coord(p2, sR, hR, R, u0[2], t.fu[2]);
    // plane q: columns along axis (1, 0, 0)[q], rows along axis (2, 2, 1)[q]
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int ca = q == 0 ? 1 : 0, ra = q == 2 ? 1 : 2;
        const Idx pi = ((Idx)q * Rp + u0[ra]) * Rp + u0[ca];
        if (!MERF_IN_RANGE(pi + Rp + 1, 3LL * Rp * Rp, kBadPlane)) {
            t.q[4 + 2 * q] = t.q[4 + 2 * q + 1] = make_uint4(0u, 0u, 0u, 0u);
            continue;
        }
        const uint4 *base = fv.planes + pi;
        t.q[4 + 2 * q] = __ldg(base);
        t.q[4 + 2 * q + 1] = __ldg(base + Rp);
    }
}

// ---------------------------------------------------------------------------------------------
// Weighted byte sums by integer dot products.  The interpolated value of channel c is
// K_c = sum_i w_i b_ic over the taps i (8 grid corners, then 4 texels per plane), and bytes are
// exact integers, so the sum is formed in integer arithmetic from fixed-point weights: the taps
// are taken in pairs (i, j), whose texel pair holds two channels as (b_ic, b_jc, b_ic', b_jc') in
// each 32-bit word, and dp2a multiplies a byte pair by a pair of 16-bit weights (w_i, w_j) and
// adds to a 32-bit accumulator, exactly.  A pair of taps and two channels cost two dot products
// per weight level, where float arithmetic needs a permute per byte, a subtraction and a
// multiply-add per two bytes.
//
// Weights.  One fused multiply-add forms each weight's last product and rounds it to the integer
// W = round(w S), S = 256 * 32767 = 2^23 - 256, in the low mantissa bits of M + w S (M = 2^23, or
// 2^23 + 128 below; the sum stays below 2^24, so the exponent byte is that of 2^23 and bit 23 is
// zero).  Byte permutes then cut the word at byte boundaries, two taps at a time: bits 8..22 form
// the high level (at most 32767) and bits 0..7 the low level, zero-extended.
// * FP32 form, every channel: M = 2^23, so the levels are H = floor(W / 256) and L = W mod 256,
//   and K_c = (256 H_c + L_c) / S exactly, with H_c, L_c the two levels' dot products.  The
//   weight's rounding (2^-24 relative to a unit weight) bounds the error of K_c by
//   20 * 255 / (2 S) < 3.1e-4 byte units, below float accumulation of the sum (half an ulp of
//   1020 per step); H_c < 20 * 32767 * 255 < 2^28.
// * 16-bit forms: M = 2^23 + 128, so the high level is H' = floor((W + 128) / 256), W / 256
//   rounded, and the low level L' = (W + 128) mod 256.  Appearance channels take the high level
//   alone, K_c = H'_c / 32767, error at most 20 * 255 * 0.502 / 32767 < 0.079 byte units
//   (typically 3e-3), within the 16-bit forms' tolerance.  Density takes both levels and the
//   tap pair's plain byte sum N_0 (one more dot product, with unit weights):
//   W + 128 = 256 H' + L', so sum_i W_i b_i0 = 256 H'_0 + L'_0 - 128 N_0, the FP32 form's integer.
// Either way density rests on the same exact integer X = sum_i W_i b_i0; the forms differ only in
// how its two parts are converted and combined in float (a few ulps of the pre-activation).
// A grid corner that is not stored holds zero bytes, so it adds nothing whatever its weight.

// c + a.h0 * b.b0 + a.h1 * b.b1 (lo) or c + a.h0 * b.b2 + a.h1 * b.b3 (hi), unsigned
__device__ __forceinline__ uint32_t dp2a_lo(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("dp2a.lo.u32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t dp2a_hi(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("dp2a.hi.u32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

constexpr float kWScale = 8388352.0f;         // S = 256 * 32767
constexpr float kWMagic = 8388608.0f;         // 2^23: H = floor(W / 256), L = W mod 256
constexpr float kWMagicRound = 8388736.0f;    // 2^23 + 128: H' = W / 256 rounded
constexpr uint32_t kSelHigh = 0x6521u;        // bytes 1, 2 of both words: bits 8..23
constexpr uint32_t kSelLow = 0xF4B0u;         // byte 0 of both words, zero-extended by the sign of byte 3

// M + round(a b): a weight's last product, rounded to an integer in the low mantissa bits.
__device__ __forceinline__ uint32_t weight_word(float a, float b, float M = kWMagic)
{
    return __float_as_uint(fmaf(a, b, M));
}

// The weights of tap pair p (taps 2p and 2p + 1, neighbours along x for the grid and along the
// column axis for a plane), scaled by S: (g, f) times the pair's shared factor v S, where
// g = 1 - f.  Grid pair p: f = f_x, v = the y and z weights of rows (p & 1, p >> 1), formed as
// w_y (w_z S) so that the two z factors serve all four pairs; plane pair p = 4 + 2q + r: plane
// q's column fraction and the weight of its row r.  The same weights as grid_w up to the
// products' association.
template <int p>
__device__ __forceinline__ void pair_factors(const Taps &t, float &f, float &vs)
{
    if constexpr (p < 4) {
        f = t.fx;
        vs = ((p & 1) ? t.fy : 1.0f - t.fy) * ((p >> 1) ? t.fz * kWScale : (1.0f - t.fz) * kWScale);
    } else {
        constexpr int q = (p - 4) >> 1, r = (p - 4) & 1;
        constexpr int ca = q == 0 ? 1 : 0, ra = q == 2 ? 1 : 2;     // column axis (1, 0, 0)[q], row axis (2, 2, 1)[q]
        f = t.fu[ca];
        vs = (r ? t.fu[ra] : 1.0f - t.fu[ra]) * kWScale;
    }
}

// Weight words of tap pair p (M + round(w S) each).
template <int p>
__device__ __forceinline__ void pair_weight_words(const Taps &t, float M, uint32_t &w0, uint32_t &w1)
{
    float f, vs;
    pair_factors<p>(t, f, vs);
    w0 = weight_word(1.0f - f, vs, M);
    w1 = weight_word(f, vs, M);
}

// Weight words (2^23 + round(w S)) of the first nt taps, all at once (the FP32 form's
// arrangement, which measured faster there than forming them pair by pair): grid corners
// trilinear, plane q bilinear in its column axis (1, 0, 0)[q] and row axis (2, 2, 1)[q].
template <int nt>
__device__ __forceinline__ void weight_words(const Taps &t, uint32_t w[nt])
{
    constexpr float S = kWScale;
    const float gx = 1.0f - t.fx, gy = 1.0f - t.fy;
    const float xy[4] = {gx * gy, t.fx * gy, gx * t.fy, t.fx * t.fy};
    const float z1 = t.fz * S, z0 = (1.0f - t.fz) * S;
#pragma unroll
    for (int c = 0; c < 8; ++c) w[c] = weight_word(xy[c & 3], (c & 4) ? z1 : z0);
    if constexpr (nt > 8) {
        const float u1[3] = {t.fu[0], t.fu[1], t.fu[2]};
        const float u0[3] = {1.0f - t.fu[0], 1.0f - t.fu[1], 1.0f - t.fu[2]};
        const float r1[3] = {0.0f, t.fu[1] * S, t.fu[2] * S};       // rows run along y or z
        const float r0[3] = {0.0f, u0[1] * S, u0[2] * S};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int ca = q == 0 ? 1 : 0, ra = q == 2 ? 1 : 2;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                w[8 + 4 * q + c] = weight_word((c & 1) ? u1[ca] : u0[ca], (c & 2) ? r1[ra] : r0[ra]);
        }
    }
}

// Integer weighted byte sums of one sample over the first nt taps.  kPrec 0 (FP32): every
// channel at two levels, K_c = (256 hi[c] + lo[c]) / S.  kPrec 1, 2 (the 16-bit forms): the
// rounded high level of every channel, hi[c] (K_c = hi[c] / 32767 for appearance), and for
// density also its low level lo[0] and byte sum n0.
template <int kPrec>
struct DotSums {
    uint32_t hi[8], lo[kPrec == 0 ? 8 : 1];
    uint32_t n0;                                 // 16-bit forms only
};

// One tap pair's contribution: its texel pair's four words are the byte pairs of channels
// (0, 1), (2, 3), (4, 5), (6, 7).  FP32: the weight words come in; 16-bit forms: the pair's words
// are formed here, just before use, so that only one pair's are live at a time.
template <int kPrec, int p>
__device__ __forceinline__ void dot_pair(const Taps &t, DotSums<kPrec> &s, const uint32_t *w)
{
    uint32_t m0, m1;
    if constexpr (kPrec == 0) {
        m0 = w[2 * p];
        m1 = w[2 * p + 1];
    } else {
        pair_weight_words<p>(t, kWMagicRound, m0, m1);
    }
    const uint32_t wh = prmt(m0, m1, kSelHigh);
    const uint32_t wl = prmt(m0, m1, kSelLow);
    const uint32_t B[4] = {t.q[p].x, t.q[p].y, t.q[p].z, t.q[p].w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        s.hi[2 * q] = dp2a_lo(wh, B[q], s.hi[2 * q]);
        s.hi[2 * q + 1] = dp2a_hi(wh, B[q], s.hi[2 * q + 1]);
        if constexpr (kPrec == 0) {
            s.lo[2 * q] = dp2a_lo(wl, B[q], s.lo[2 * q]);
            s.lo[2 * q + 1] = dp2a_hi(wl, B[q], s.lo[2 * q + 1]);
        }
    }
    if constexpr (kPrec != 0) {
        s.lo[0] = dp2a_lo(wl, B[0], s.lo[0]);
        s.n0 = dp2a_lo(0x00010001u, B[0], s.n0);
    }
}

template <int kPrec, int nt>
__device__ __forceinline__ void dot_sums(const Taps &t, DotSums<kPrec> &s)
{
#pragma unroll
    for (int c = 0; c < 8; ++c) s.hi[c] = 0u;
#pragma unroll
    for (int c = 0; c < (kPrec == 0 ? 8 : 1); ++c) s.lo[c] = 0u;
    s.n0 = 0u;
    uint32_t w[kPrec == 0 ? nt : 1];
    if constexpr (kPrec == 0) weight_words<nt>(t, w);
    dot_pair<kPrec, 0>(t, s, w);
    dot_pair<kPrec, 1>(t, s, w);
    dot_pair<kPrec, 2>(t, s, w);
    dot_pair<kPrec, 3>(t, s, w);
    if constexpr (nt > 8) {
        dot_pair<kPrec, 4>(t, s, w);
        dot_pair<kPrec, 5>(t, s, w);
        dot_pair<kPrec, 6>(t, s, w);
        dot_pair<kPrec, 7>(t, s, w);
        dot_pair<kPrec, 8>(t, s, w);
        dot_pair<kPrec, 9>(t, s, w);
    }
}

// Density pre-activation: (28 / 255) K_0 - 14 W, where W = W_V + 3 is the total interpolation
// weight of the sources (the planes' weights sum to one each; W = W_V for a grid-only scene), and
// K_0 = X / S with X = sum_i W_i b_i0 = 256 H_0 + L_0 (FP32) = 128 (2 H'_0 - N_0) + L'_0 (16-bit
// forms).  The low parts convert exactly (< 2^21); the high parts round only above 2^24.  Every
// path of one form that evaluates a uint8 scene's density calls this one expression, so their
// opacities agree bit for bit.
template <int kPrec>
__device__ __forceinline__ float dequant_density(const DotSums<kPrec> &k, float wsum)
{
    constexpr float A = 28.0f / 255.0f;
    if constexpr (kPrec == 0)
        return fmaf(__uint2float_rn(k.lo[0]), A * (1.0f / kWScale),
                    fmaf(__uint2float_rn(k.hi[0]), A * (256.0f / kWScale), -14.0f * wsum));
    else
        return fmaf(__uint2float_rn(k.lo[0]), A * (1.0f / kWScale),
                    fmaf(__int2float_rn((int)(2u * k.hi[0]) - (int)k.n0), A * (128.0f / kWScale), -14.0f * wsum));
}

// Dense float storage: all eight channels of all 20 taps, summed.
template <int kGeo = kGeoRuntime>
__device__ __forceinline__ void field_f32(const FieldView &fv, float p0, float p1, float p2, float out[8])
{
    using Idx = typename GatherIndex<kGeo>::T;
    const float sL = (float)fv.L * 0.25f;
    const int hL = fv.L >> 1, L = fv.L;
    int x0, y0, z0;
    float fx, fy, fz;
    texel_coord(p0, sL, hL, L, x0, fx);
    texel_coord(p1, sL, hL, L, y0, fy);
    texel_coord(p2, sL, hL, L, z0, fz);
    // eight channels as four packed FP32 pairs (each lane rounds as the scalar fmaf does)
    float2 acc[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = make_float2(0.0f, 0.0f);
    const Idx gidx = ((Idx)z0 * L + y0) * L + x0;
    const bool g_ok = MERF_IN_RANGE(gidx + (Idx)L * L + L + 1, (long long)L * L * L, kBadDense);
    const float4 *g0 = fv.grid_f32 + gidx * 2;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
        const float w = (cx ? fx : 1.0f - fx) * (cy ? fy : 1.0f - fy) * (cz ? fz : 1.0f - fz);
        const float4 *q = g0 + ((Idx)(cz * L + cy) * L + cx) * 2;
        if (!g_ok) continue;
        const float4 a = __ldg(q), b = __ldg(q + 1);
        const float2 ww = make_float2(w, w);
        acc[0] = __ffma2_rn(ww, make_float2(a.x, a.y), acc[0]);
        acc[1] = __ffma2_rn(ww, make_float2(a.z, a.w), acc[1]);
        acc[2] = __ffma2_rn(ww, make_float2(b.x, b.y), acc[2]);
        acc[3] = __ffma2_rn(ww, make_float2(b.z, b.w), acc[3]);
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
        const Idx pidx = ((Idx)q * R + u0[ra]) * R + u0[ca];
        if (!MERF_IN_RANGE(pidx + R + 1, 3LL * R * R, kBadDense)) continue;
        const float4 *t0 = fv.planes_f32 + pidx * 2;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int cu = c & 1, cv = c >> 1;
            const float w = (cu ? fu[ca] : 1.0f - fu[ca]) * (cv ? fu[ra] : 1.0f - fu[ra]);
            const float4 *t = t0 + ((Idx)cv * R + cu) * 2;
            const float4 a = __ldg(t), b = __ldg(t + 1);
            const float2 ww = make_float2(w, w);
            acc[0] = __ffma2_rn(ww, make_float2(a.x, a.y), acc[0]);
            acc[1] = __ffma2_rn(ww, make_float2(a.z, a.w), acc[1]);
            acc[2] = __ffma2_rn(ww, make_float2(b.x, b.y), acc[2]);
            acc[3] = __ffma2_rn(ww, make_float2(b.z, b.w), acc[3]);
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        out[2 * j] = acc[j].x;
        out[2 * j + 1] = acc[j].y;
    }
}

}  // namespace merf
