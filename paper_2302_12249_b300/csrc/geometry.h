// geometry.h -- which compiled gather variant renders a scene: the host's choice, in plain C++ (no
// device code), shared by the C-ABI translation units and the kernels' template parameters.
//
// kGeoRuntime reads L, B and R from the FieldView.  kGeoPaper is the paper's configuration (L = 512
// stored in 16^3 blocks, planes R = 2048; Sec. 4), for which every stride, shift and scale of the
// gather is a compile-time constant and every atlas, plane and occupancy offset is 32-bit.
// kGeoGridOnly is a scene with no planes (R = 0, t~ = V: the SNeRG++-style baseline the paper
// compares against in Sec. 6), L and B read at run time, offsets 32-bit; kGeoGridOnlyWide is the
// same gather with 64-bit offsets, for grid-only scenes whose offsets do not fit 32 bits.  Dense
// float scenes (the differentiable storage) take kGeoDense32, 32-bit offsets, when theirs fit, and
// kGeoRuntime (64-bit) otherwise.
#pragma once

#include "merf.h"

namespace merf {

constexpr int kGeoRuntime = 0, kGeoPaper = 1, kGeoGridOnly = 2, kGeoGridOnlyWide = 3, kGeoDense32 = 4;
template <int kGeo>
constexpr bool kGridOnly = kGeo == kGeoGridOnly || kGeo == kGeoGridOnlyWide;

// Largest finest occupancy level whose cell offsets the 32-bit variants take: 1024^3 cells.
constexpr int kMaxOccRes32 = 1024;

// True when every offset of a uint8 scene fits 32 bits: the largest atlas voxel offset,
// n_blocks (B + 1)^3 - 1 (blocks carry a one-voxel apron), and the largest finest occupancy cell
// offset, N^3 - 1 with N <= kMaxOccRes32.  (The paper geometry's plane offsets stay below
// 3 * 2050^2; grid-only scenes have no planes.)
inline bool offsets_fit_32(const merf_scene_desc &d)
{
    const unsigned long long b1 = (unsigned long long)d.block_size + 1;
    return d.n_blocks >= 0 && (unsigned long long)d.n_blocks * b1 * b1 * b1 <= 0xffffffffull &&
           d.n_occ_levels >= 1 && d.occ_res[0] <= kMaxOccRes32;
}

// True when every offset of a dense float scene fits 32 bits as a signed value, counted in floats:
// the grid holds L^3 texels of 8 floats (8 L^3 float offsets; the forward pass addresses them as
// 2 L^3 float4, the adjoint's gradient scatter as 8 floats per texel), the planes 3 R^2 texels
// (24 R^2 floats), and the finest occupancy level at most kMaxOccRes32^3 cells.  So L <= 645 and
// R <= 9459.
inline bool dense_offsets_fit_32(const merf_scene_desc &d)
{
    const unsigned long long L = (unsigned long long)d.grid_res, R = (unsigned long long)d.plane_res;
    return d.grid_res >= 0 && d.plane_res >= 0 && 8ull * L * L * L <= 0x7fffffffull &&
           24ull * R * R <= 0x7fffffffull && d.n_occ_levels >= 1 && d.occ_res[0] <= kMaxOccRes32;
}

// True when the gather may use the kernels compiled for the paper's geometry (kGeoPaper): its
// sizes, and offsets that fit 32 bits.
inline bool paper_geometry(const merf_scene_desc &d)
{
    return d.storage == MERF_STORAGE_U8_SPARSE && d.grid_res == 512 && d.block_size == 16 && d.plane_res == 2048 &&
           offsets_fit_32(d);
}

// The gather variant of a scene: the paper's geometry, a grid-only uint8 scene (no planes; 32- or
// 64-bit offsets), a dense float scene with 32-bit offsets, or run-time strides.
inline int gather_geometry(const merf_scene_desc &d)
{
    if (d.storage == MERF_STORAGE_F32_DENSE) return dense_offsets_fit_32(d) ? kGeoDense32 : kGeoRuntime;
    if (paper_geometry(d)) return kGeoPaper;
    if (d.storage == MERF_STORAGE_U8_SPARSE && d.plane_res == 0)
        return offsets_fit_32(d) ? kGeoGridOnly : kGeoGridOnlyWide;
    return kGeoRuntime;
}

}  // namespace merf
