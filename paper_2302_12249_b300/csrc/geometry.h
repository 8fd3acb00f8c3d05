// geometry.h -- which compiled gather variant renders a scene: the host's choice, in plain C++ (no
// device code), shared by the C-ABI translation units and the kernels' template parameters.
//
// kGeoRuntime reads L, B and R from the FieldView.  kGeoPaper is the paper's configuration (L = 512
// stored in 16^3 blocks, planes R = 2048; Sec. 4), for which every stride, shift and scale of the
// gather is a compile-time constant and every atlas, plane and occupancy offset is 32-bit.
// kGeoGridOnly is a scene with no planes (R = 0, t~ = V: the SNeRG++-style baseline the paper
// compares against in Sec. 6), L and B read at run time.
#pragma once

#include "merf.h"

namespace merf {

constexpr int kGeoRuntime = 0, kGeoPaper = 1, kGeoGridOnly = 2;

// Largest atlas, in blocks of 17^3 voxels (16^3 plus the apron), whose voxel offsets fit 32 bits.
constexpr unsigned long long kPaperMaxBlocks = 0xffffffffull / (17ull * 17ull * 17ull);
// Largest finest occupancy level of a paper-geometry scene: 1024^3 cells, offsets below 2^30.
constexpr int kPaperMaxOccRes = 1024;

// True when the gather may use the kernels compiled for the paper's geometry (kGeoPaper): its
// sizes, at most kPaperMaxBlocks atlas blocks and a finest occupancy level of at most
// kPaperMaxOccRes^3 cells, so that every offset fits 32 bits.
inline bool paper_geometry(const merf_scene_desc &d)
{
    return d.storage == MERF_STORAGE_U8_SPARSE && d.grid_res == 512 && d.block_size == 16 && d.plane_res == 2048 &&
           d.n_blocks >= 0 && (unsigned long long)d.n_blocks <= kPaperMaxBlocks && d.n_occ_levels >= 1 &&
           d.occ_res[0] <= kPaperMaxOccRes;
}

// The gather variant of a scene: the paper's geometry, a grid-only uint8 scene (no planes), or
// run-time strides.
inline int gather_geometry(const merf_scene_desc &d)
{
    if (paper_geometry(d)) return kGeoPaper;
    if (d.storage == MERF_STORAGE_U8_SPARSE && d.plane_res == 0) return kGeoGridOnly;
    return kGeoRuntime;
}

}  // namespace merf
