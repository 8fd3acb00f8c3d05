// scene.h -- library-internal definition of a resident scene and its device views (shared by the
// C-ABI translation units; not part of the public interface).
#pragma once

#include <cuda_runtime.h>

#include "geometry.h"
#include "merf.h"
#include "render.cuh"

struct merf_scene {
    merf_scene_desc desc;
    int device;
    void *index_grid = nullptr, *atlas = nullptr, *planes = nullptr, *mlp = nullptr;
    void *occ[MERF_MAX_OCC_LEVELS] = {};
    size_t bytes = 0;
    unsigned long long param_version = 0;   // parameter installs: upload 0, +1 per merf_scene_set_dense
};

namespace merf {

inline int log2_int(int v)
{
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

// Field and occupancy views of a resident scene, as the kernels read them.
inline void scene_views(const merf_scene *s, FieldView &fv, OccView &occ)
{
    const merf_scene_desc &d = s->desc;
    fv = FieldView{};
    fv.L = d.grid_res;
    fv.R = d.plane_res;
    if (d.storage == MERF_STORAGE_U8_SPARSE) {
        fv.B = d.block_size;
        fv.log2B = log2_int(d.block_size);
        fv.nb = d.grid_res / d.block_size;
        fv.n_blocks = d.n_blocks;
        fv.index_grid = (const int32_t *)s->index_grid;
        fv.atlas = (const uint4 *)s->atlas;
        fv.planes = (const uint4 *)s->planes;
    } else {
        fv.grid_f32 = (const float4 *)s->atlas;
        fv.planes_f32 = (const float4 *)s->planes;
    }
    occ = OccView{};
    occ.n = d.n_occ_levels;
    for (int l = 0; l < d.n_occ_levels; ++l) {
        occ.level[l] = (const uint8_t *)s->occ[l];
        occ.res[l] = d.occ_res[l];
        occ.shift[l] = log2_int(d.occ_res[0] / d.occ_res[l]);
    }
}

// Bounds-checked build: read and clear the server translation unit's device status word (0 in
// the release build).
unsigned int take_server_status();

// Thread-local error message of the C ABI (defined in merf_api.cu).
merf_status set_error(merf_status s, const char *fmt, ...);
merf_status clear_error();

}  // namespace merf
