// debug.cuh -- index checks of the bounds-checked build (compiled with -DMERF_DEBUG_BOUNDS).
//
// In that build every data-dependent index into the index grid, the atlas, the planes, the
// occupancy levels and the dense float arrays is checked before the access.  An index out of
// range sets a bit of the translation unit's device status word and the access is skipped (the
// texel reads as zero, the cell as empty); nothing traps.  The host reads and clears the word
// with merf_check_device.  In the release build MERF_IN_RANGE is the constant true and the checks
// compile to nothing.
#pragma once

#include <cuda_runtime.h>

namespace merf {

enum : unsigned {
    kBadIndexGrid = 1u,   // index-grid entry
    kBadAtlas = 2u,       // atlas voxel
    kBadPlane = 4u,       // plane texel
    kBadOcc = 8u,         // occupancy cell
    kBadDense = 16u,      // dense float grid or plane texel (or its gradient)
    kStatusSelfTest = 1u << 31,
};

#ifdef MERF_DEBUG_BOUNDS
static __device__ unsigned int g_status;   // one per translation unit

__device__ __forceinline__ bool in_range(long long i, long long n, unsigned bit)
{
    if (i >= 0 && i < n) return true;
    atomicOr(&g_status, bit);
    return false;
}
#define MERF_IN_RANGE(i, n, bit) ::merf::in_range((long long)(i), (long long)(n), (bit))
#else
#define MERF_IN_RANGE(i, n, bit) true
#endif

}  // namespace merf
