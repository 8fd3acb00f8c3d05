// debug.cuh -- the device status word: bounded waits that gave up (every build) and, in the
// bounds-checked build (compiled with -DMERF_DEBUG_BOUNDS), out-of-range indices.
//
// In that build every data-dependent index into the index grid, the atlas, the planes, the
// occupancy levels and the dense float arrays is checked before the access.  An index out of
// range sets a bit of the translation unit's device status word and the access is skipped (the
// texel reads as zero, the cell as empty); nothing traps.  In the release build MERF_IN_RANGE is
// the constant true and the checks compile to nothing.  A wait on the MLP weights' bulk copy or on
// the tensor cores' completion barrier that runs out of polls sets kWaitTimeout in both builds.
// The host reads and clears the word with merf_check_device.
#pragma once

#include <cuda_runtime.h>

namespace merf {

enum : unsigned {
    kBadIndexGrid = 1u,   // index-grid entry
    kBadAtlas = 2u,       // atlas voxel
    kBadPlane = 4u,       // plane texel
    kBadOcc = 8u,         // occupancy cell
    kBadDense = 16u,      // dense float grid or plane texel (or its gradient)
    kWaitTimeout = 32u,   // a bounded device-side wait gave up
    kStatusSelfTest = 1u << 31,
};

static __device__ unsigned int g_status;   // one per translation unit

__device__ __forceinline__ void set_status(unsigned bit) { atomicOr(&g_status, bit); }

#ifdef MERF_DEBUG_BOUNDS
__device__ __forceinline__ bool in_range(long long i, long long n, unsigned bit)
{
    if (i >= 0 && i < n) return true;
    set_status(bit);
    return false;
}
#define MERF_IN_RANGE(i, n, bit) ::merf::in_range((long long)(i), (long long)(n), (bit))
#else
#define MERF_IN_RANGE(i, n, bit) true
#endif

}  // namespace merf
