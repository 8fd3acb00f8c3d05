// Host-side entry to the gather-variant choice (geometry.h), for the CPU tests: no device code.
#include "geometry.h"

extern "C" int host_gather_geometry(const merf_scene_desc *d) { return merf::gather_geometry(*d); }
extern "C" int host_offsets_fit_32(const merf_scene_desc *d) { return merf::offsets_fit_32(*d) ? 1 : 0; }
