/* merf.h -- C ABI of the B300 renderer for baked MERF scenes.
 *
 * Renders the baked representation of "MERF: Memory-Efficient Radiance Fields for
 * Real-time View Synthesis in Unbounded Scenes" (Reiser et al. 2023): per pixel ray, the
 * piecewise-projective contraction (Sec. 3.2), empty-space skipping against a max-pooled
 * occupancy hierarchy (Sec. 5), the summed tri/bilinear uint8 feature field (Sec. 3.1,
 * Sec. 4.2), front-to-back compositing with early termination (Eq. 1, Eq. 2, Sec. 5) and
 * the deferred view-dependence MLP (Sec. 2, App. B).
 *
 * Conventions shared by every entry point
 *   - Device work is enqueued on the caller's CUDA stream (`stream`, a cudaStream_t; NULL =
 *     legacy default stream).  merf_render, merf_render_aux and merf_trace allocate nothing
 *     and do not synchronise, so they may be captured into a CUDA graph; the upload, free
 *     and host-output calls synchronise as documented.
 *   - Pointers documented as "device" must be device memory of the current device;
 *     "host" pointers are read before the call returns and may be freed afterwards.
 *   - No C++ exception crosses this boundary.  Every call returns a merf_status; on
 *     failure merf_last_error() holds a message for the calling thread and no device work
 *     was enqueued (argument checks happen before any launch).
 *
 * Coordinates: contracted space is [-2, 2]^3.  Every array of resolution N samples it at
 * texel centres p_i = (i + 1/2) 4/N - 2; lookups clamp to the edge texel.  3D arrays are
 * indexed [z][y][x] (x fastest) with the C = 8 channels innermost: channel 0 density,
 * 1..3 diffuse RGB, 4..7 the view-dependence feature (Sec. 3.1).
 */
#ifndef MERF_H
#define MERF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum merf_status {
    MERF_OK = 0,
    MERF_ERR_INVALID_ARG = 1,   /* a pointer, size, layout or option is invalid */
    MERF_ERR_OOM = 2,           /* device allocation failed or exceeds the device budget */
    MERF_ERR_CUDA = 3,          /* a CUDA runtime call failed (message in merf_last_error) */
    MERF_ERR_TIMEOUT = 4,       /* a bounded wait expired (merf_server_wait) */
    MERF_ERR_DEVICE_BOUNDS = 5, /* a kernel detected an out-of-range index and skipped it */
    MERF_ERR_UNSUPPORTED = 6,   /* a valid request this build does not implement */
    MERF_ERR_CANCELLED = 7      /* the server request was withdrawn by merf_server_cancel */
} merf_status;

enum { MERF_STORAGE_U8_SPARSE = 0, MERF_STORAGE_F32_DENSE = 1 };
enum { MERF_PREC_FP32 = 0, MERF_PREC_FP16 = 1, MERF_PREC_BF16 = 2 };
enum { MERF_MAX_OCC_LEVELS = 8 };
enum { MERF_CHANNELS = 8, MERF_MLP_IN = 34, MERF_MLP_HIDDEN = 16, MERF_MLP_OUT = 3 };
/* 34*16 + 16 + 16*16 + 16 + 16*3 + 3 */
enum { MERF_MLP_PARAMS = 883 };
/* per-pixel diagnostic record written by merf_render_aux (floats) */
enum {
    MERF_AUX_CD = 0,      /* [3] accumulated diffuse colour C_d (Eq. 2) */
    MERF_AUX_F = 3,       /* [4] accumulated feature F (Eq. 2) */
    MERF_AUX_T = 7,       /* transmittance after the last composited sample */
    MERF_AUX_NLAT = 8,    /* lattice samples on the ray */
    MERF_AUX_NEVAL = 9,   /* samples evaluated (occupied, before termination) */
    MERF_AUX_NAPP = 10,   /* evaluated samples with non-zero opacity (appearance read) */
    MERF_AUX_TERM = 11,   /* 1 if the ray stopped by early termination */
    MERF_AUX_SIZE = 12
};
/* device counters accumulated by merf_render_aux (uint64) */
enum { MERF_CNT_RAYS = 0, MERF_CNT_LATTICE = 1, MERF_CNT_EVAL = 2, MERF_CNT_APPEAR = 3,
       MERF_CNT_SIZE = 4 };

/* A pinhole camera (OpenCV axes: x right, y down, z forward).  c2w is the row-major 3x4
 * camera-to-world matrix [R | o]; the ray of pixel column i, row j leaves o through
 * ((i + 1/2 - cx)/fx, (j + 1/2 - cy)/fy, 1) in camera coordinates. */
typedef struct merf_camera {
    float c2w[12];
    float fx, fy, cx, cy;
} merf_camera;

/* Shape of a baked scene (Sec. 3.1, Sec. 4.3, Sec. 5). */
typedef struct merf_scene_desc {
    int32_t grid_res;        /* L: 3D grid resolution; even, a multiple of block_size */
    int32_t block_size;      /* B: block edge in voxels, a power of two (sparse storage) */
    int32_t plane_res;       /* R: resolution of the three planes; even.  0 (uint8 storage only):
                                a grid-only scene, t~ = V -- the SNeRG++-style baseline that
                                Sec. 6 compares MERF with; `planes` is then ignored (may be NULL) */
    int32_t channels;        /* C: must be 8 */
    int32_t n_blocks;        /* stored blocks in the atlas (sparse storage) */
    int32_t n_occ_levels;    /* 1 .. MERF_MAX_OCC_LEVELS */
    int32_t occ_res[MERF_MAX_OCC_LEVELS]; /* finest first; powers of two >= 2, each dividing
                                              the previous; coarser levels are max-pools */
    int32_t mlp_in, mlp_hidden, mlp_out;  /* must be 34, 16, 3 */
    int32_t storage;         /* MERF_STORAGE_U8_SPARSE or MERF_STORAGE_F32_DENSE */
} merf_scene_desc;

typedef struct merf_render_opts {
    float step;          /* lattice step delta_s in contracted arc length, > 0 */
    float t_term;        /* early-termination threshold on transmittance (Sec. 5: 2e-4) */
    int32_t precision;   /* MERF_PREC_FP32: every step in FP32.  MERF_PREC_FP16 / _BF16 (uint8
                            storage only): appearance interpolated with 15-bit fixed-point
                            weights, appearance sigmoids through tanh.approx, and the deferred MLP
                            on the tcgen05 tensor cores (16-bit operands, FP32 accumulation);
                            density is the FP32 form's exact integer sum (converted to float in a
                            different order: a few ulps), and opacity, transmittance, compositing
                            and traversal stay FP32, so the evaluated samples are the FP32
                            form's */
    int32_t early_term;  /* 1: stop a ray after the sample at which T < t_term */
    int32_t contraction; /* 0: contract_pi (Sec. 3.2) with its segment lattice and empty-space
                            skipping.  1: the ablation of Sec. 3.2 / Table 2 (c), mip-NeRF 360's
                            spherical contraction (Eq. contract360): rays bend, so every sample of
                            a dense march -- s_k = (k + 1/2) step for (k + 1) step < 2, ray
                            parameter t(s) = s (s <= 1), 1/(2 - s) beyond -- is visited and
                            evaluated iff its finest occupancy cell is set.  FP32 only; not for
                            merf_render_backward (MERF_ERR_UNSUPPORTED). */
} merf_render_opts;

typedef struct merf_scene merf_scene;  /* opaque; owns device memory */

/* Copy a baked scene to the device (Sec. 4.3: block-sparse 3D grid, three planes,
 * occupancy hierarchy, deferred-MLP weights).  Host arrays (read before return):
 *   index_grid  int32 [(L/B)^3]            block id in [0, n_blocks) or -1 (not stored)
 *   atlas       uint8 [n_blocks][B][B][B][8]
 *   planes      uint8 [3][R][R][8]         P_x(y,z) [z][y], P_y(x,z) [z][x], P_z(x,y) [y][x]
 *                                          (NULL allowed when plane_res is 0: grid only)
 *   occ_levels  n_occ_levels pointers to uint8 [N][N][N], non-zero = occupied
 *   mlp_weights float32 [883]: W0[34][16], b0[16], W1[16][16], b1[16], W2[16][3], b2[3]
 * On the device the weights become one 11,776-byte block: the FP32 weights, then the FP16 and
 * BF16 forms packed as the tensor cores read them (built by a kernel on `stream`).  The atlas
 * (with a one-voxel apron per block) and the planes (with a one-texel border) are stored as
 * 16-byte texel pairs along x (along u for a plane), the two texels' bytes interleaved: about
 * twice the texel bytes of the baked arrays, so that the renderer needs no byte permutes.
 * The layout is validated (ids in range, every coarse occupancy cell that is empty has
 * only empty children) before anything is allocated.  Returns MERF_ERR_OOM without
 * touching the device if the scene exceeds the budget set by merf_set_device_budget.
 * Synchronises `stream` before returning.  *out receives a handle owned by the caller,
 * released with merf_scene_free. */
merf_status merf_scene_upload(const merf_scene_desc *desc, const int32_t *index_grid,
                              const uint8_t *atlas, const uint8_t *planes,
                              const uint8_t *const *occ_levels, const float *mlp_weights,
                              void *stream, merf_scene **out);

/* merf_scene_upload with the scene's arrays in device memory (on the current device, the same
 * layouts as merf_scene_upload: index_grid int32 [(L/B)^3], atlas uint8 [n_blocks][B][B][B][8],
 * planes uint8 [3][R][R][8] or NULL when R = 0, occupancy levels uint8 [N][N][N] (an array of
 * device pointers in host memory), mlp float32 [883]).  For scenes too large to stage in host
 * memory, or already on the GPU (Sec. 4.3's baked arrays produced there): the index grid,
 * occupancy levels and MLP weights (a few MB) are copied to the host and checked as
 * merf_scene_upload checks them, and, in addition, every atlas slot must be named by exactly one
 * index-grid entry; the padded atlas and bordered planes are built by kernels on `stream` from
 * the caller's arrays, which the call only reads.  Synchronises `stream` before returning; the
 * caller may free its arrays then.  Errors as merf_scene_upload. */
merf_status merf_scene_upload_device(const merf_scene_desc *desc, const int32_t *d_index_grid,
                                     const uint8_t *d_atlas, const uint8_t *d_planes,
                                     const uint8_t *const *d_occ_levels, const float *d_mlp, void *stream,
                                     merf_scene **out);

/* Same for a dense float32 scene (storage MERF_STORAGE_F32_DENSE): grid float32
 * [L][L][L][8] and planes float32 [3][R][R][8] hold pre-activation values directly
 * (no dequantisation); block_size and n_blocks are ignored. */
merf_status merf_scene_upload_dense(const merf_scene_desc *desc, const float *grid,
                                    const float *planes, const uint8_t *const *occ_levels,
                                    const float *mlp_weights, void *stream, merf_scene **out);

/* Release a scene (NULL is ignored).  Synchronises the device first. */
void merf_scene_free(merf_scene *scene);

/* Device bytes held by a scene (its arrays in the device layout plus the 11,776-byte MLP
 * block). */
size_t merf_scene_device_bytes(const merf_scene *scene);

/* Scene files: one baked scene as a raw binary file -- the arrays merf_scene_upload(_dense) takes,
 * behind a 256-byte header, all little-endian.  After the header each array starts at the next
 * multiple of 64 bytes, in this order:
 *   uint8 storage:  index_grid int32 [(L/B)^3], atlas uint8 [n_blocks][B][B][B][8],
 *                   planes uint8 [3][R][R][8] (absent when R = 0);
 *   float storage:  grid float32 [L][L][L][8], planes float32 [3][R][R][8];
 *   then both:      occupancy levels uint8 [N_l][N_l][N_l] (finest first), MLP float32 [883].
 * The file ends at the end of the MLP. */
typedef struct merf_scene_file_header {
    char magic[8];               /* "MERFSCN1" */
    uint32_t version;            /* 1 */
    uint32_t header_bytes;       /* 256 */
    uint64_t file_bytes;         /* size of the whole file */
    float step;                  /* lattice step the scene was made for (informational) */
    int32_t seed;                /* generator seed (informational) */
    char name[32];               /* NUL-padded name (informational) */
    merf_scene_desc desc;        /* as for merf_scene_upload(_dense) */
    uint8_t reserved[120];       /* zero */
} merf_scene_file_header;

/* Map a scene file and upload it: merf_scene_upload or merf_scene_upload_dense on its arrays, with
 * their validation, results and errors (asynchronous on `stream` in the same way).
 * MERF_ERR_INVALID_ARG if the file cannot be opened or mapped, its magic, version or header size
 * is not the format's, its descriptor is invalid or has more blocks than the index grid, or its
 * size differs from the one its descriptor implies. */
merf_status merf_scene_load(const char *path, void *stream, merf_scene **out);

/* Render n_cams images of W x H pixels into `out` (device float32 [n_cams][H][W][3],
 * written, never read): C = C_d + h(C_d, F, d) per pixel (Sec. 2).  `cams` is a host array
 * of n_cams cameras.  Asynchronous on `stream`, with no allocation and no synchronisation, so it
 * can be captured into a CUDA graph; the cameras travel by value in the kernel parameters, so a
 * captured graph replays the cameras it was captured with. */
merf_status merf_render(const merf_scene *scene, const merf_camera *cams, int n_cams, int W,
                        int H, float *out, const merf_render_opts *opts, void *stream);

/* merf_render plus optional diagnostics: `aux` (device float32 [n_cams][H][W][MERF_AUX_SIZE]
 * or NULL) and `counters` (device uint64 [MERF_CNT_SIZE] or NULL, accumulated with atomics:
 * the caller zeroes it). */
merf_status merf_render_aux(const merf_scene *scene, const merf_camera *cams, int n_cams, int W,
                            int H, float *out, float *aux, unsigned long long *counters,
                            const merf_render_opts *opts, void *stream);

/* Render into host memory `h_out` (host float32 [n_cams][H][W][3]).  If h_out is page-locked
 * memory the device can address (cudaHostAlloc, or cudaHostRegister'ed, under unified
 * addressing) the kernel writes the image there directly in one launch; `d_staging` is unused
 * and may be NULL.  Otherwise the call renders like merf_render into the caller's device buffer
 * `d_staging` (same shape), one launch per camera on `stream`, while the previous camera's image
 * is copied to h_out on a library-owned copy stream (created on the first call on each device).
 * Returns when the image is in h_out. */
merf_status merf_render_host(const merf_scene *scene, const merf_camera *cams, int n_cams,
                             int W, int H, float *d_staging, float *h_out,
                             const merf_render_opts *opts, void *stream);

/* Like merf_render_host, but the caller passes no device buffer and the call allocates none.
 * The paper has no counterpart; this is a service for callers that cannot allocate device
 * memory themselves, for example an application whose own memory manager owns the whole device
 * pool, or a per-frame render loop that must not call cudaMalloc because it can synchronise the
 * device and stall other work.  The image is rendered into a fixed device staging area that
 * is part of the library (MERF_NOALLOC_STAGING_BYTES = 32 MiB, enough for one 1920x1080 RGB
 * float frame; every GPU that loads the library holds it until the process exits) and copied to
 * `h_out` (host float32 [n_cams][H][W][3]; page-locked for the copy to be asynchronous).
 * Requests whose image exceeds the staging area return MERF_ERR_INVALID_ARG.  The first call
 * on a device looks up the staging area's device address (cudaGetSymbolAddress) with that
 * device current.  All calls share the one staging area: the kernel writes every pixel of it
 * that the call returns, so nothing needs clearing, but calls that overlap on the GPU (from
 * several host threads or streams at once) race on it.  Returns after the copy has completed. */
enum { MERF_NOALLOC_STAGING_BYTES = 32 << 20 };
merf_status merf_render_host_noalloc(const merf_scene *scene, const merf_camera *cams, int n_cams,
                                     int W, int H, float *h_out, const merf_render_opts *opts,
                                     void *stream);

/* Evaluated-sample sets of the traversal alone (Sec. 5 empty-space skipping, early
 * termination off): bit k of mask row r (device uint32 [n_cams*H*W][words], row
 * r = (cam*H + row)*W + col) is set iff lattice sample k of that ray lies in an occupied
 * finest occupancy cell; bits beyond 32*words are dropped.  n_lattice (device int32
 * [n_cams*H*W]) receives the number of lattice samples per ray. */
merf_status merf_trace(const merf_scene *scene, const merf_camera *cams, int n_cams, int W,
                       int H, uint32_t *mask, int words, int32_t *n_lattice,
                       const merf_render_opts *opts, void *stream);

/* Replace the parameters of a dense float scene (storage MERF_STORAGE_F32_DENSE) with new values
 * from device memory: grid float32 [L][L][L][8], planes float32 [3][R][R][8], mlp float32 [883]
 * (device-to-device copies on `stream`, and the MLP's 16-bit forms rebuilt by a kernel there; no
 * allocation).  Used between optimisation steps. */
merf_status merf_scene_set_dense(merf_scene *scene, const float *d_grid, const float *d_planes,
                                 const float *d_mlp, void *stream);

/* How many times merf_scene_set_dense has replaced this scene's parameters (0 after upload; 0 for a
 * NULL scene).  The adjoint differentiates at the parameters the scene holds when it runs, so a
 * caller that keeps a forward pass for a later backward records this count at the forward and,
 * if it has changed, installs that forward's parameters again before the adjoint (the Python
 * autograd wrapper does so).  Host only, no synchronisation: the count changes when the copies
 * are queued. */
unsigned long long merf_scene_param_version(const merf_scene *scene);

/* Adjoint of merf_render for dense float scenes in FP32 (Eq. 1, Eq. 2, Sec. 3.1, App. B): given
 * d_out = dL/dC (device float32 [n_cams][H][W][3]), accumulate dL/dgrid, dL/dplanes and dL/dmlp
 * into g_grid, g_planes, g_mlp (device, shapes of merf_scene_set_dense's arguments; the caller
 * zeroes them).  Lattice, occupancy and early-termination decisions are those of the forward
 * pass with the same cameras and options (they do not depend on the parameters except through
 * termination).  Transmittance is recomputed by a second front-to-back march, not stored.
 * Gradient sums use atomics, so results vary in the last bits between runs. */
merf_status merf_render_backward(const merf_scene *scene, const merf_camera *cams, int n_cams, int W, int H,
                                 const float *d_out, float *g_grid, float *g_planes, float *g_mlp,
                                 const merf_render_opts *opts, void *stream);

/* merf_render_backward without the recomputed forward march: `aux` is the per-pixel record
 * (device float32 [n_cams][H][W][MERF_AUX_SIZE]) that merf_render_aux wrote for the same scene
 * parameters, cameras and options; its C_d and F stand in for the first march.  NULL: as
 * merf_render_backward.  The paper has no counterpart (it trains through other means). */
merf_status merf_render_backward_aux(const merf_scene *scene, const merf_camera *cams, int n_cams, int W, int H,
                                     const float *d_out, const float *aux, float *g_grid, float *g_planes,
                                     float *g_mlp, const merf_render_opts *opts, void *stream);

/* ----------------------------------------------------------------------------------------
 * Serving: a render server holding several resident scenes and batching requests of mixed
 * scenes and resolutions continuously.  The paper renders one view at a time in a browser; this
 * is the serving form built around its renderer (Sec. 5).
 *
 * A server thread admits submitted requests in arrival order when the request's output image
 * fits in the free part of the server's device output pool (admission by memory), then packs
 * pixel tiles (16 x 8) of all admitted requests -- oldest first, across scenes and resolutions --
 * into iterations of at most max_tiles_per_iter tiles.  Each iteration is one launch of a captured
 * CUDA graph: work-list upload, counter reset, and a persistent kernel whose CTAs take tiles from
 * the list with an atomic counter.  Two iterations are kept in flight, so requests that arrive
 * while the GPU is busy join the next iteration and their tiles share launches with the
 * requests already running.  A finished request's image is copied to its host buffer on a copy
 * stream; it completes when that copy has landed.  No device-side wait exists: every kernel
 * terminates on its own once the tile list is exhausted.  A request not yet being copied out can
 * be cancelled; its pool space is released once no iteration in flight can still write it. */
typedef struct merf_server merf_server;

typedef struct merf_server_opts {
    size_t pool_bytes;            /* device output pool (admission limit), >= one request */
    int32_t max_tiles_per_iter;   /* tiles of 16 x 8 pixels per iteration, 1 .. 65536 */
    int32_t precision;            /* MERF_PREC_*, as in merf_render_opts */
    float step;                   /* lattice step, as in merf_render_opts */
    float t_term;                 /* early-termination threshold */
    int32_t early_term;
    int32_t max_tiles_backlog;    /* 0, or max_tiles_per_iter .. 65536: tiles an iteration may carry
                                     while more than twice max_tiles_per_iter tiles of admitted and
                                     queued requests wait to be scheduled (fewer, larger iterations
                                     under load; 0 keeps every iteration at max_tiles_per_iter) */
} merf_server_opts;

typedef struct merf_server_stats {
    unsigned long long submitted, completed, rays, iterations, tiles;
    unsigned long long cancelled;         /* requests withdrawn by merf_server_cancel */
    size_t pool_bytes, peak_pool_bytes;   /* pool size and its peak reservation */
    size_t pool_used_bytes;               /* reserved now (admitted requests, cancelled ones in flight) */
    int32_t peak_admitted;                /* most requests admitted at once */
    int32_t admitted;                     /* requests holding pool space now */
    int32_t queued;                       /* requests waiting for admission now */
    int32_t reserved;
} merf_server_stats;

/* Create a server over n_scenes (1..8) scenes uploaded with merf_scene_upload (uint8 storage) on
 * the current device; the scenes must outlive the server.  Allocates the output pool, the
 * work-list buffers and two captured graphs, and starts the server thread. */
merf_status merf_server_create(const merf_scene *const *scenes, int n_scenes, const merf_server_opts *opts,
                               merf_server **out);

/* Submit one request: render scene `scene` from camera *cam (host, copied) at W x H into h_out
 * (host float32 [H][W][3], page-locked for the copy to be asynchronous; written when the request
 * completes).  Returns at once with *req_id.  MERF_ERR_OOM if the image alone exceeds the pool. */
merf_status merf_server_submit(merf_server *srv, int scene, const merf_camera *cam, int W, int H, float *h_out,
                               uint64_t *req_id);

/* Block until request req_id completes (or timeout_s elapses: MERF_ERR_TIMEOUT, the request
 * stays pending and may be waited for again).  On completion *latency_s (may be NULL) receives
 * the time from submission to the image being in host memory, and the request is released: wait
 * once per request.  A cancelled request returns MERF_ERR_CANCELLED (latency: to its release), one
 * that failed on the device MERF_ERR_CUDA. */
merf_status merf_server_wait(merf_server *srv, uint64_t req_id, double timeout_s, double *latency_s);

/* Where a request's latency went, in seconds (host clock, sampled by the server thread, which
 * polls every 50 us at most): admit_s from submission to admission by pool memory, queue_s from
 * admission to the launch of the first iteration carrying its tiles, render_s from there to the
 * completion of the last iteration carrying its tiles, copy_s from there to the image in host
 * memory.  The four add up to total_s, the latency merf_server_wait reports. */
typedef struct merf_request_timing {
    double total_s, admit_s, queue_s, render_s, copy_s;
} merf_request_timing;

/* merf_server_wait that also fills *timing (may be NULL) on completion. */
merf_status merf_server_wait_timed(merf_server *srv, uint64_t req_id, double timeout_s, double *latency_s,
                                   merf_request_timing *timing);

/* Withdraw request req_id.  *cancelled = 1 if it was still waiting for admission or rendering
 * (its tiles may still be running): from this call on, its h_out is never written, and
 * merf_server_wait returns MERF_ERR_CANCELLED once no iteration in flight carries its tiles (its
 * pool space is free again then).  *cancelled = 0 if its image is already being copied out or it
 * has completed: it finishes normally.  MERF_ERR_INVALID_ARG for an unknown (or already waited
 * for) request.  The request must still be waited for, once, to release it. */
merf_status merf_server_cancel(merf_server *srv, uint64_t req_id, int *cancelled);

merf_status merf_server_get_stats(merf_server *srv, merf_server_stats *out);

/* Finish every submitted request, stop the thread and release the server (NULL is ignored). */
void merf_server_destroy(merf_server *srv);

/* Device-memory budget for merf_scene_upload* (bytes; 0 = unlimited, the default). */
void merf_set_device_budget(size_t bytes);

/* Synchronise `stream` and report the device status word.  In the bounds-checked build
 * (libmerf_debug.so, compiled with MERF_DEBUG_BOUNDS) every kernel checks each data-dependent
 * index into the index grid, atlas, planes, occupancy levels and dense arrays; an index out of
 * range is skipped (the texel reads as zero, the cell as empty) and recorded, never trapped.
 * Returns MERF_ERR_DEVICE_BOUNDS (merf_last_error names what was out of range) if anything was
 * recorded since the last call, and clears the word.  In every build the render and serving
 * kernels wait for the bulk copy of the MLP weights, and the FP16/BF16 kernels for their
 * tensor-core MMAs, on barriers with a bounded number of polls; a wait that gives up (the MLP term
 * of its pixels is then unreliable; after an MMA wait it reads as zero) is recorded too, and
 * reported as MERF_ERR_TIMEOUT.
 * self_test exercises the reporting paths first: 1 (bounds-checked build only, else
 * MERF_ERR_UNSUPPORTED) records a self-test bit from a one-thread kernel (the call returns
 * MERF_ERR_DEVICE_BOUNDS); 2 (any build) runs the MLP's bounded barrier wait on a barrier that
 * nothing arrives on, which gives up after 1000 polls (the call returns MERF_ERR_TIMEOUT). */
merf_status merf_check_device(void *stream, int self_test);

/* Message of the last failed call on this thread ("" if none). */
const char *merf_last_error(void);

/* Library version string. */
const char *merf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MERF_H */
