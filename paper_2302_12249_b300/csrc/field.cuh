// field.cuh -- the MERF feature field at a contracted point (Sec. 3.1, Sec. 4.2) for sm_103a.
//
// t~(p) = V(x, y, z) + P_x(y, z) + P_y(x, z) + P_z(x, y): trilinear interpolation in the
// low-resolution 3D grid plus bilinear interpolation in three high-resolution planes, each
// texel dequantised as 2 m k / 255 - m (m = 14 for density, 7 otherwise).  Because the
// dequantisation is affine and interpolation weights sum to one, the kernel interpolates raw
// byte values and dequantises the sum once per channel:
//     t~_c = (2 m_c / 255) * sum_w w k_c  -  m_c * (W_V + 3),
// with W_V the weight of the 3D-grid corners that are stored (a voxel of a block that is not
// stored contributes nothing).  A grid-only scene (no planes, R = 0: the SNeRG++-style baseline
// of Sec. 6) has t~ = V and the offset m_c W_V.
//
// Layout in HBM.  Every texel is 8 bytes (one uint2: channels 0..3 in .x, 4..7 in .y), so a
// single 64-bit load fetches density and appearance of a corner.  The 3D grid is
// block-sparse: an int32 index grid over (L/B)^3 blocks holds, for a stored block, its atlas
// slot in bits 0..23 and in bits 24..30 a mask of which of its +x/+y/+z neighbour blocks are
// not stored (neighbour dx + 2 dy + 4 dz in 1..7 at bit 23 + that number); -1 marks a block
// that is not stored.  Each atlas slot holds (B+1)^3 voxels [z][y][x]: the block plus a
// one-voxel apron copied from its +x/+y/+z neighbours, so the eight corners of any sample
// whose lowest corner lies in the block are one base address plus constant offsets.
// For the 3D grid, clamp-to-edge is folded into the integer coordinate and weight (lowest corner
// kept in [0, N-2]), so no lookup leaves the array.  The planes are stored [3][R+2][R+2] with a
// one-texel border that repeats their edge texels, so their taps need no clamp.  The occupancy
// grids are not read here (the traversal tests them before a sample is evaluated).
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
    const uint2 *atlas;          // [n_blocks][B+1][B+1][B+1]
    const uint2 *planes;         // [3][R+2][R+2]: one-texel clamp-to-edge border
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

// Byte b of a 32-bit word as a float: the byte is placed in the low mantissa bits of 2^23
// (one byte permute) and 2^23 is subtracted; both steps are exact.
template <int b>
__device__ __forceinline__ float byte_f(uint32_t w)
{
    return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u | b)) - 8388608.0f;
}

template <int c>
__device__ __forceinline__ float byte_of(uint2 v)
{
    return c < 4 ? byte_f<c & 3>(v.x) : byte_f<c & 3>(v.y);
}

// The 20 texels of one sample (8 grid corners, 4 texels in each plane) and their weights.
struct Taps {
    uint2 v[20];
    float fx, fy, fz;       // grid fractions
    float fu[3];            // plane fractions along x, y, z
    float wv;               // weight of the stored grid corners
};

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

__device__ __forceinline__ float plane_w(const Taps &t, int q, int c)
{
    const int ca = q == 0 ? 1 : 0, ra = q == 2 ? 1 : 2;
    return ((c & 1) ? t.fu[ca] : 1.0f - t.fu[ca]) * ((c & 2) ? t.fu[ra] : 1.0f - t.fu[ra]);
}

// Lowest corner in a block that is not stored: every corner is looked up on its own.
__device__ __forceinline__ void gather_grid_slow(const FieldView &fv, int x0, int y0, int z0, Taps &t)
{
    const int sh = fv.log2B, msk = fv.B - 1, nb = fv.nb, B1 = fv.B + 1;
    uint32_t gmask = 0u;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int x = x0 + (c & 1), y = y0 + ((c >> 1) & 1), z = z0 + (c >> 2);
        const int gi = ((z >> sh) * nb + (y >> sh)) * nb + (x >> sh);
        const int ent = MERF_IN_RANGE(gi, nb * nb * nb, kBadIndexGrid) ? __ldg(fv.index_grid + gi) : -1;
        const size_t slot = (size_t)(ent & 0xffffff);
        const size_t ai = ((slot * B1 + (z & msk)) * B1 + (y & msk)) * B1 + (x & msk);
        if (ent >= 0 && MERF_IN_RANGE(ai, (long long)fv.n_blocks * B1 * B1 * B1, kBadAtlas)) {
            t.v[c] = __ldg(fv.atlas + ai);
            gmask |= 1u << c;
        } else {
            t.v[c] = make_uint2(0u, 0u);
        }
    }
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
            for (int c = 0; c < 8; ++c) t.v[c] = make_uint2(0u, 0u);
            t.wv = 0.0f;
            goto grid_done;
        }
        const uint2 *base = fv.atlas + ai;
        const int sy = B1, sz = B1 * B1;
        t.v[0] = __ldg(base);
        t.v[1] = __ldg(base + 1);
        t.v[2] = __ldg(base + sy);
        t.v[3] = __ldg(base + sy + 1);
        t.v[4] = __ldg(base + sz);
        t.v[5] = __ldg(base + sz + 1);
        t.v[6] = __ldg(base + sz + sy);
        t.v[7] = __ldg(base + sz + sy + 1);
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
            t.v[8 + 4 * q + 0] = t.v[8 + 4 * q + 1] = t.v[8 + 4 * q + 2] = t.v[8 + 4 * q + 3] = make_uint2(0u, 0u);
            continue;
        }
        const uint2 *base = fv.planes + pi;
        t.v[8 + 4 * q + 0] = __ldg(base);
        t.v[8 + 4 * q + 1] = __ldg(base + 1);
        t.v[8 + 4 * q + 2] = __ldg(base + Rp);
        t.v[8 + 4 * q + 3] = __ldg(base + Rp + 1);
    }
}

// Density pre-activation from its weighted byte sum k: (28 / 255) k - 14 W, where W = W_V + 3
// is the total interpolation weight of the sources (the planes' weights sum to one each; W = W_V
// for a grid-only scene).  Every path that evaluates density calls this one expression, so their
// opacities agree bit for bit.
__device__ __forceinline__ float dequant_density(float k, float wsum)
{
    return k * (28.0f / 255.0f) - 14.0f * wsum;
}


// Bytes b and b + 1 of a 32-bit word as two floats (byte_f on both, the subtraction packed).
template <int b>
__device__ __forceinline__ float2 byte_pair_f(uint32_t w)
{
    const float2 m = make_float2(__uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u | b)),
                                 __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u | (b + 1))));
    return __fadd2_rn(m, make_float2(-8388608.0f, -8388608.0f));
}

// All eight pre-activations in one pass over the taps (tap-major): each tap's weight is formed
// once and its eight bytes are accumulated into four running float2 sums with packed FP32
// arithmetic (each lane rounds exactly as the scalar fmaf does).
template <int i>
__device__ __forceinline__ void accumulate_tap(const Taps &t, float2 acc[4])
{
    const float w = i < 8 ? grid_w(t, i) : plane_w(t, (i - 8) >> 2, (i - 8) & 3);
    const float2 ww = make_float2(w, w);
    acc[0] = __ffma2_rn(ww, byte_pair_f<0>(t.v[i].x), acc[0]);
    acc[1] = __ffma2_rn(ww, byte_pair_f<2>(t.v[i].x), acc[1]);
    acc[2] = __ffma2_rn(ww, byte_pair_f<0>(t.v[i].y), acc[2]);
    acc[3] = __ffma2_rn(ww, byte_pair_f<2>(t.v[i].y), acc[3]);
}

// Weighted byte sums of all eight channels, as the pairs (0, 1), (2, 3), (4, 5), (6, 7), over
// the first nt taps (20: grid and planes; 8: grid only).
template <int nt = 20>
__device__ __forceinline__ void byte_sums_u8(const Taps &t, float2 acc[4])
{
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = make_float2(0.0f, 0.0f);
    accumulate_tap<0>(t, acc);  accumulate_tap<1>(t, acc);  accumulate_tap<2>(t, acc);
    accumulate_tap<3>(t, acc);  accumulate_tap<4>(t, acc);  accumulate_tap<5>(t, acc);
    accumulate_tap<6>(t, acc);  accumulate_tap<7>(t, acc);
    if constexpr (nt > 8) {
        accumulate_tap<8>(t, acc);  accumulate_tap<9>(t, acc);  accumulate_tap<10>(t, acc);
        accumulate_tap<11>(t, acc); accumulate_tap<12>(t, acc); accumulate_tap<13>(t, acc);
        accumulate_tap<14>(t, acc); accumulate_tap<15>(t, acc); accumulate_tap<16>(t, acc);
        accumulate_tap<17>(t, acc); accumulate_tap<18>(t, acc); accumulate_tap<19>(t, acc);
    }
}

// ---------------------------------------------------------------------------------------------
// Reduced-precision byte sums (the precision form).  Density and channel 1 keep the FP32 packed
// pair of the FP32 path (so density, opacity and transmittance are those of the FP32 path bit
// for bit); channels (2, 3), (4, 5), (6, 7) go through 16-bit pairs.  Within each source (grid,
// P_x, P_y, P_z) every tap is taken relative to the source's first tap: the difference of two
// bytes is an exact integer in [-255, 255] (exact in half and in bfloat16), so the 16-bit
// arithmetic only carries the interpolation corrections sum_i w_i (b_i - b_first), with weights
// rounded to that type.  A grid corner that is not stored holds zero bytes, so with the
// unmasked trilinear weights summing to one the first taps enter with weight one; their sum is
// an integer <= 1020, exact in either form:
//     K_c = b_first,V + b_first,Px + b_first,Py + b_first,Pz + sum of corrections.
// FP16: one byte permute gives a half2 of 1024 + byte for two channels (the half 0x64XX is
// 1024 + XX), and the difference of two such halves is the exact byte difference.  BF16 (7
// stored mantissa bits cannot hold 1024 + byte) takes the differences in FP32 from the packed
// 2^23 + byte floats; their high halves are their exact bfloat16 values.

__device__ __forceinline__ __half2 magic_h2(uint32_t w, uint32_t sel)
{
    const uint32_t u = __byte_perm(w, 0x64646464u, sel);
    __half2 h;
    memcpy(&h, &u, 4);
    return h;
}

// 2^23 + byte for bytes b and b + 1 of a word (no subtraction).
template <int b>
__device__ __forceinline__ float2 byte_pair_magic(uint32_t w)
{
    return make_float2(__uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u | b)),
                       __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u | (b + 1))));
}

template <int kPrec>
struct LpAcc;
template <>
struct LpAcc<1> {                        // FP16
    __half2 first[3], fsum[3], corr[3];
};
template <>
struct LpAcc<2> {                        // BF16
    float2 nfirst[3], fsum[3];           // nfirst: -(2^23 + first byte)
    __nv_bfloat162 corr[3];
};

template <int kPrec, int i>
__device__ __forceinline__ void lp_tap(const Taps &t, float2 &k01, LpAcc<kPrec> &a)
{
    constexpr bool first = i == 0 || i == 8 || i == 12 || i == 16;
    const float w = i < 8 ? grid_w(t, i) : plane_w(t, (i - 8) >> 2, (i - 8) & 3);
    k01 = __ffma2_rn(make_float2(w, w), byte_pair_f<0>(t.v[i].x), k01);
    if constexpr (kPrec == 1) {
        const __half2 m[3] = {magic_h2(t.v[i].x, 0x4342u), magic_h2(t.v[i].y, 0x4140u),
                              magic_h2(t.v[i].y, 0x4342u)};
        if constexpr (first) {
            const __half2 mag = __float2half2_rn(1024.0f);
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                a.first[p] = m[p];
                a.fsum[p] = i == 0 ? __hsub2(m[p], mag) : __hadd2(a.fsum[p], __hsub2(m[p], mag));
            }
        } else {
            const __half2 w2 = __float2half2_rn(w);
#pragma unroll
            for (int p = 0; p < 3; ++p) a.corr[p] = __hfma2(w2, __hsub2(m[p], a.first[p]), a.corr[p]);
        }
    } else {
        const float2 m[3] = {byte_pair_magic<2>(t.v[i].x), byte_pair_magic<0>(t.v[i].y),
                             byte_pair_magic<2>(t.v[i].y)};
        if constexpr (first) {
            const float2 nmag = make_float2(-8388608.0f, -8388608.0f);
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                a.nfirst[p] = make_float2(-m[p].x, -m[p].y);
                a.fsum[p] = i == 0 ? __fadd2_rn(m[p], nmag) : __fadd2_rn(a.fsum[p], __fadd2_rn(m[p], nmag));
            }
        } else {
            const __nv_bfloat162 w2 = __float2bfloat162_rn(w);
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                // d holds exact integers |d| <= 255, which bfloat16 keeps exactly; a bfloat16 is
                // the high half of the FP32 word, so one byte permute packs the pair
                const float2 d = __fadd2_rn(m[p], a.nfirst[p]);
                const uint32_t u = __byte_perm(__float_as_uint(d.x), __float_as_uint(d.y), 0x7632u);
                __nv_bfloat162 db;
                memcpy(&db, &u, 4);
                a.corr[p] = __hfma2(w2, db, a.corr[p]);
            }
        }
    }
}

// Weighted byte sums in the layout of byte_sums_u8: k[0] = channels (0, 1) in FP32, k[1..3] =
// channels (2, 3), (4, 5), (6, 7) from their 16-bit corrections.
template <int kPrec, int nt = 20>
__device__ __forceinline__ void byte_sums_lp(const Taps &t, float2 k[4])
{
    LpAcc<kPrec> a;
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        if constexpr (kPrec == 1) a.corr[p] = __float2half2_rn(0.0f);
        else a.corr[p] = __float2bfloat162_rn(0.0f);
    }
    k[0] = make_float2(0.0f, 0.0f);
    lp_tap<kPrec, 0>(t, k[0], a);  lp_tap<kPrec, 1>(t, k[0], a);  lp_tap<kPrec, 2>(t, k[0], a);
    lp_tap<kPrec, 3>(t, k[0], a);  lp_tap<kPrec, 4>(t, k[0], a);  lp_tap<kPrec, 5>(t, k[0], a);
    lp_tap<kPrec, 6>(t, k[0], a);  lp_tap<kPrec, 7>(t, k[0], a);
    if constexpr (nt > 8) {
        lp_tap<kPrec, 8>(t, k[0], a);  lp_tap<kPrec, 9>(t, k[0], a);  lp_tap<kPrec, 10>(t, k[0], a);
        lp_tap<kPrec, 11>(t, k[0], a); lp_tap<kPrec, 12>(t, k[0], a); lp_tap<kPrec, 13>(t, k[0], a);
        lp_tap<kPrec, 14>(t, k[0], a); lp_tap<kPrec, 15>(t, k[0], a); lp_tap<kPrec, 16>(t, k[0], a);
        lp_tap<kPrec, 17>(t, k[0], a); lp_tap<kPrec, 18>(t, k[0], a); lp_tap<kPrec, 19>(t, k[0], a);
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        if constexpr (kPrec == 1) k[1 + p] = __fadd2_rn(__half22float2(a.fsum[p]), __half22float2(a.corr[p]));
        else k[1 + p] = __fadd2_rn(a.fsum[p], __bfloat1622float2(a.corr[p]));
    }
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
