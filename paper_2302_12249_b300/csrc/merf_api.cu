// merf_api.cu -- the C ABI declared in include/merf.h: scene upload/validation, argument
// checks and kernel launches.  Host code only; the device code is in render.cuh.
#include <cuda_runtime.h>
#include <errno.h>
#include <fcntl.h>
#include <sys/mman.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "merf.h"
#include "backward.cuh"
#include "render.cuh"
#include "nvtx.h"
#include "scene.h"

namespace {

thread_local std::string g_err;
size_t g_budget = 0;

merf_status fail(merf_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

merf_status ok()
{
    g_err.clear();
    return MERF_OK;
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

merf_status check_desc(const merf_scene_desc *d, int storage)
{
    if (!d) return fail(MERF_ERR_INVALID_ARG, "desc is NULL");
    if (d->storage != storage)
        return fail(MERF_ERR_INVALID_ARG, "desc->storage %d does not match the upload call", d->storage);
    if (d->channels != MERF_CHANNELS) return fail(MERF_ERR_INVALID_ARG, "channels must be 8, got %d", d->channels);
    if (d->mlp_in != MERF_MLP_IN || d->mlp_hidden != MERF_MLP_HIDDEN || d->mlp_out != MERF_MLP_OUT)
        return fail(MERF_ERR_UNSUPPORTED, "MLP %d->%d->%d not supported (34->16->16->3 only)", d->mlp_in,
                    d->mlp_hidden, d->mlp_out);
    if (d->grid_res < 2 || d->grid_res > 4096 || (d->grid_res & 1))
        return fail(MERF_ERR_INVALID_ARG, "grid_res %d must be even in [2, 4096]", d->grid_res);
    // plane_res 0: a grid-only scene (uint8 storage only), the SNeRG++-style baseline of Sec. 6
    const bool grid_only = storage == MERF_STORAGE_U8_SPARSE && d->plane_res == 0;
    if (!grid_only && (d->plane_res < 2 || d->plane_res > 16384 || (d->plane_res & 1)))
        return fail(MERF_ERR_INVALID_ARG, "plane_res %d must be even in [2, 16384] (or 0 for a grid-only uint8 scene)",
                    d->plane_res);
    if (storage == MERF_STORAGE_U8_SPARSE) {
        if (!pow2(d->block_size) || d->block_size > d->grid_res || d->grid_res % d->block_size)
            return fail(MERF_ERR_INVALID_ARG, "block_size %d must be a power of two dividing grid_res %d",
                        d->block_size, d->grid_res);
        if (d->n_blocks < 0) return fail(MERF_ERR_INVALID_ARG, "n_blocks %d < 0", d->n_blocks);
        if (d->grid_res / d->block_size > 1024)
            return fail(MERF_ERR_INVALID_ARG, "grid_res / block_size = %d exceeds 1024 blocks per axis",
                        d->grid_res / d->block_size);
    }
    if (d->n_occ_levels < 1 || d->n_occ_levels > MERF_MAX_OCC_LEVELS)
        return fail(MERF_ERR_INVALID_ARG, "n_occ_levels %d not in [1, %d]", d->n_occ_levels, MERF_MAX_OCC_LEVELS);
    for (int l = 0; l < d->n_occ_levels; ++l) {
        int n = d->occ_res[l];
        if (!pow2(n) || n < 2 || n > 4096)
            return fail(MERF_ERR_INVALID_ARG, "occ_res[%d] = %d must be a power of two in [2, 4096]", l, n);
        if (l > 0 && (n >= d->occ_res[l - 1]))
            return fail(MERF_ERR_INVALID_ARG, "occ_res must decrease from finest to coarsest");
    }
    return MERF_OK;
}

// Every empty cell of a coarser level must have only empty children in the finest level
// (max-pooling, Sec. 5); otherwise skipping would drop occupied samples.
merf_status check_occupancy(const merf_scene_desc *d, const uint8_t *const *occ)
{
    if (!occ) return fail(MERF_ERR_INVALID_ARG, "occ_levels is NULL");
    for (int l = 0; l < d->n_occ_levels; ++l)
        if (!occ[l]) return fail(MERF_ERR_INVALID_ARG, "occ_levels[%d] is NULL", l);
    const int N0 = d->occ_res[0];
    for (int l = 1; l < d->n_occ_levels; ++l) {
        const int Nl = d->occ_res[l], f = N0 / Nl;
        for (int z = 0; z < N0; ++z)
            for (int y = 0; y < N0; ++y)
                for (int x = 0; x < N0; ++x) {
                    if (!occ[0][((size_t)z * N0 + y) * N0 + x]) continue;
                    if (!occ[l][((size_t)(z / f) * Nl + y / f) * Nl + x / f])
                        return fail(MERF_ERR_INVALID_ARG,
                                    "occupancy level %d cell (%d,%d,%d) is empty but finest cell (%d,%d,%d) is set",
                                    l, x / f, y / f, z / f, x, y, z);
                }
    }
    return MERF_OK;
}

static_assert(merf::kMlpBlockBytes == 11776, "the MLP block size merf.h states");

// Fill the FP16 and BF16 forms of a scene's MLP block from its FP32 weights (one CTA).
__global__ void __launch_bounds__(merf::kThreads) mlp_pack_kernel(uint8_t *block)
{
    const float *w = reinterpret_cast<const float *>(block);
    merf::mlp_pack16<1>(*reinterpret_cast<merf::MlpWeights16<1> *>(block + merf::kMlpOffF16), w);
    merf::mlp_pack16<2>(*reinterpret_cast<merf::MlpWeights16<2> *>(block + merf::kMlpOffBf16), w);
}

// The MLP block from n FP32 weights at src (host or device memory, `kind`): zero it, copy the
// weights in, pack the 16-bit forms; all on `st`.
cudaError_t put_mlp_block(void *block, const float *src, cudaMemcpyKind kind, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(block, 0, merf::kMlpBlockBytes, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(block, src, sizeof(float) * MERF_MLP_PARAMS, kind, st);
    if (e != cudaSuccess) return e;
    mlp_pack_kernel<<<1, merf::kThreads, 0, st>>>((uint8_t *)block);
    return cudaGetLastError();
}

void free_scene_memory(merf_scene *s)
{
    cudaFree(s->index_grid);
    cudaFree(s->atlas);
    cudaFree(s->planes);
    cudaFree(s->mlp);
    for (auto &p : s->occ) cudaFree(p);
}

merf_status upload_common(const merf_scene_desc *desc, const void *grid, size_t grid_bytes,
                          const void *planes, size_t plane_bytes, const int32_t *index_grid,
                          size_t index_bytes, const uint8_t *const *occ, const float *mlp,
                          void *stream, merf_scene **out)
{
    size_t occ_bytes[MERF_MAX_OCC_LEVELS] = {};
    size_t total = grid_bytes + plane_bytes + index_bytes + merf::kMlpBlockBytes;
    for (int l = 0; l < desc->n_occ_levels; ++l) {
        occ_bytes[l] = (size_t)desc->occ_res[l] * desc->occ_res[l] * desc->occ_res[l];
        total += occ_bytes[l];
    }
    if (g_budget && total > g_budget)
        return fail(MERF_ERR_OOM, "scene needs %zu device bytes, budget is %zu", total, g_budget);
    merf_scene *s = new merf_scene();
    s->desc = *desc;
    cudaGetDevice(&s->device);
    cudaStream_t st = (cudaStream_t)stream;
    struct Item { void **dst; const void *src; size_t n; };
    std::vector<Item> items = {{&s->atlas, grid, grid_bytes},
                               {&s->planes, planes, plane_bytes},
                               {&s->index_grid, index_grid, index_bytes},
                               {&s->mlp, nullptr, merf::kMlpBlockBytes}};
    for (int l = 0; l < desc->n_occ_levels; ++l) items.push_back({&s->occ[l], occ[l], occ_bytes[l]});
    for (auto &it : items) {
        if (it.n == 0) continue;
        cudaError_t e = cudaMalloc(it.dst, it.n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            free_scene_memory(s);
            delete s;
            return fail(e == cudaErrorMemoryAllocation ? MERF_ERR_OOM : MERF_ERR_CUDA,
                        "cudaMalloc(%zu): %s", it.n, cudaGetErrorString(e));
        }
        e = it.dst == &s->mlp ? put_mlp_block(s->mlp, mlp, cudaMemcpyHostToDevice, st)
                              : cudaMemcpyAsync(*it.dst, it.src, it.n, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            free_scene_memory(s);
            delete s;
            return fail(MERF_ERR_CUDA, "cudaMemcpyAsync: %s", cudaGetErrorString(e));
        }
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        free_scene_memory(s);
        delete s;
        return fail(MERF_ERR_CUDA, "upload: %s", cudaGetErrorString(e));
    }
    s->bytes = total;
    *out = s;
    return ok();
}

merf_status check_opts(const merf_render_opts *o)
{
    if (!o) return fail(MERF_ERR_INVALID_ARG, "opts is NULL");
    if (!(o->step > 0.0f) || !std::isfinite(o->step) || o->step < 1e-5f)
        return fail(MERF_ERR_INVALID_ARG, "step %g must be finite and >= 1e-5", (double)o->step);
    if (!(o->t_term >= 0.0f) || !(o->t_term < 1.0f))
        return fail(MERF_ERR_INVALID_ARG, "t_term %g must be in [0, 1)", (double)o->t_term);
    if (o->early_term != 0 && o->early_term != 1)
        return fail(MERF_ERR_INVALID_ARG, "early_term must be 0 or 1");
    if (o->contraction != 0 && o->contraction != 1)
        return fail(MERF_ERR_INVALID_ARG, "contraction %d must be 0 (contract_pi) or 1 (spherical)", o->contraction);
    if (o->contraction == 1 && o->precision != MERF_PREC_FP32)
        return fail(MERF_ERR_UNSUPPORTED, "the spherical-contraction ablation renders in FP32 only");
    if (o->precision != MERF_PREC_FP32 && o->precision != MERF_PREC_FP16 && o->precision != MERF_PREC_BF16)
        return fail(MERF_ERR_INVALID_ARG, "precision %d is not a MERF_PREC_* value", o->precision);
    return MERF_OK;
}

merf_status check_frame(const merf_scene *s, const merf_camera *cams, int n, int W, int H)
{
    if (!s) return fail(MERF_ERR_INVALID_ARG, "scene is NULL");
    if (!cams) return fail(MERF_ERR_INVALID_ARG, "cams is NULL");
    if (n < 1 || W < 1 || H < 1) return fail(MERF_ERR_INVALID_ARG, "n_cams %d, W %d, H %d must be >= 1", n, W, H);
    if (W > 16384 || H > 16384) return fail(MERF_ERR_INVALID_ARG, "W %d / H %d exceed 16384", W, H);
    if ((double)n * W * H > 2.0e9) return fail(MERF_ERR_INVALID_ARG, "n_cams * W * H exceeds 2e9 rays");
    for (int c = 0; c < n; ++c) {
        const merf_camera &k = cams[c];
        for (int t = 0; t < 12; ++t)
            if (!std::isfinite(k.c2w[t])) return fail(MERF_ERR_INVALID_ARG, "camera %d c2w not finite", c);
        if (!(std::fabs(k.fx) > 0.0f) || !(std::fabs(k.fy) > 0.0f) || !std::isfinite(k.fx) ||
            !std::isfinite(k.fy) || !std::isfinite(k.cx) || !std::isfinite(k.cy))
            return fail(MERF_ERR_INVALID_ARG, "camera %d intrinsics invalid", c);
    }
    return MERF_OK;
}

merf::RenderParams make_params(const merf_scene *s, const merf_render_opts *o, int W, int H)
{
    merf::RenderParams P;
    memset(&P, 0, sizeof P);
    merf::scene_views(s, P.fv, P.occ);
    P.mlp = (const float *)s->mlp;
    P.W = W;
    P.H = H;
    P.step = o->step;
    P.t_term = o->t_term;
    P.early_term = o->early_term;
    P.contraction = o->contraction;
    return P;
}

#ifdef MERF_DEBUG_BOUNDS
__global__ void status_self_test_kernel() { atomicOr(&merf::g_status, merf::kStatusSelfTest); }
#endif

// A bounded wait that runs out: an mbarrier that nothing arrives on, waited on for 100 us of the
// global timer with the same wait the tensor-core MLP uses; giving up is recorded as the MLP's
// would be.
__global__ void wait_timeout_self_test_kernel()
{
    __shared__ alignas(8) uint64_t mbar;
    merf::mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!merf::mbar_wait(&mbar, 0, 100000)) merf::set_status(merf::kWaitTimeout);
}

template <int kPrec>
void launch_u8(int geo, dim3 grid, dim3 block, cudaStream_t st, const merf::RenderParams &P)
{
    if (geo == merf::kGeoPaper)
        merf::render_kernel<0, kPrec, merf::kGeoPaper><<<grid, block, 0, st>>>(P);
    else if (geo == merf::kGeoGridOnly)
        merf::render_kernel<0, kPrec, merf::kGeoGridOnly><<<grid, block, 0, st>>>(P);
    else if (geo == merf::kGeoGridOnlyWide)
        merf::render_kernel<0, kPrec, merf::kGeoGridOnlyWide><<<grid, block, 0, st>>>(P);
    else
        merf::render_kernel<0, kPrec, merf::kGeoRuntime><<<grid, block, 0, st>>>(P);
}

merf_status launch_render(const merf_scene *s, const merf_camera *cams, int n, int W, int H, float *out,
                          float *aux, unsigned long long *counters, const merf_render_opts *o,
                          cudaStream_t st)
{
    if (o->precision != MERF_PREC_FP32 && s->desc.storage != MERF_STORAGE_U8_SPARSE)
        return fail(MERF_ERR_UNSUPPORTED, "reduced precision needs uint8 block-sparse storage");
    merf::RenderParams P = make_params(s, o, W, H);
    P.out = out;
    P.aux = aux;
    P.counters = counters;
    const dim3 block(merf::kThreads);
    for (int c0 = 0; c0 < n; c0 += merf::kMaxCams) {
        const int nc = std::min(merf::kMaxCams, n - c0);
        P.cam0 = c0;
        for (int c = 0; c < nc; ++c) memcpy(P.cams.m[c], &cams[c0 + c], sizeof(merf_camera));
        const dim3 grid((W + merf::kTileW - 1) / merf::kTileW, (H + merf::kTileH - 1) / merf::kTileH, nc);
        const int geo = merf::gather_geometry(s->desc);
        if (o->contraction == 1) {          // spherical-contraction ablation (FP32, dense march)
            if (geo == merf::kGeoDense32)
                merf::render_kernel<1, 0, merf::kGeoDense32, 1><<<grid, block, 0, st>>>(P);
            else if (s->desc.storage == MERF_STORAGE_F32_DENSE)
                merf::render_kernel<1, 0, merf::kGeoRuntime, 1><<<grid, block, 0, st>>>(P);
            else if (geo == merf::kGeoPaper)
                merf::render_kernel<0, 0, merf::kGeoPaper, 1><<<grid, block, 0, st>>>(P);
            else if (geo == merf::kGeoGridOnly)
                merf::render_kernel<0, 0, merf::kGeoGridOnly, 1><<<grid, block, 0, st>>>(P);
            else if (geo == merf::kGeoGridOnlyWide)
                merf::render_kernel<0, 0, merf::kGeoGridOnlyWide, 1><<<grid, block, 0, st>>>(P);
            else
                merf::render_kernel<0, 0, merf::kGeoRuntime, 1><<<grid, block, 0, st>>>(P);
        } else if (geo == merf::kGeoDense32)
            merf::render_kernel<1, 0, merf::kGeoDense32><<<grid, block, 0, st>>>(P);
        else if (s->desc.storage == MERF_STORAGE_F32_DENSE)
            merf::render_kernel<1, 0, merf::kGeoRuntime><<<grid, block, 0, st>>>(P);
        else if (o->precision == MERF_PREC_FP16)
            launch_u8<1>(geo, grid, block, st, P);
        else if (o->precision == MERF_PREC_BF16)
            launch_u8<2>(geo, grid, block, st, P);
        else
            launch_u8<0>(geo, grid, block, st, P);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(MERF_ERR_CUDA, "render launch: %s", cudaGetErrorString(e));
    }
    return ok();
}

}  // namespace

namespace merf {
merf_status set_error(merf_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}
merf_status clear_error() { return ok(); }
}  // namespace merf

// The device index grid: a stored block's atlas slot in bits 0..23 and, in bits 24..30, a mask of
// its +x/+y/+z neighbour blocks (dx + 2 dy + 4 dz in 1..7, bit 23 + that number) that are not
// stored or lie past the grid edge; -1 for a block that is not stored.
static std::vector<int32_t> index_with_neighbour_masks(const int32_t *index_grid, size_t nbi)
{
    std::vector<int32_t> ig(nbi * nbi * nbi);
    auto id_at = [&](size_t bx, size_t by, size_t bz) -> int32_t {
        if (bx >= nbi || by >= nbi || bz >= nbi) return -1;
        return index_grid[(bz * nbi + by) * nbi + bx];
    };
    for (size_t bz = 0; bz < nbi; ++bz)
        for (size_t by = 0; by < nbi; ++by)
            for (size_t bx = 0; bx < nbi; ++bx) {
                const int32_t id = id_at(bx, by, bz);
                if (id < 0) { ig[(bz * nbi + by) * nbi + bx] = -1; continue; }
                uint32_t miss = 0;
                for (int n = 1; n < 8; ++n)
                    if (id_at(bx + (n & 1), by + ((n >> 1) & 1), bz + (n >> 2)) < 0) miss |= 1u << (n - 1);
                ig[(bz * nbi + by) * nbi + bx] = (int32_t)((uint32_t)id | (miss << 24));
            }
    return ig;
}

// The padded atlas from an unpadded one in device memory: CTA `slot` fills the (B+1)^3 voxels of
// that atlas slot (the block at `coords[slot]` = bx | by << 10 | bz << 20, plus its +x/+y/+z apron
// from the neighbouring blocks; zero where a neighbour is not stored or past the grid edge), each
// stored as the texel pair (x, x + 1) with the two texels' bytes interleaved (pair_bytes); the
// pair of the last column has a zero upper texel.  index_grid: the caller's grid (slot or -1),
// already validated.
__global__ void pad_atlas_kernel(const uint2 *atlas, const int32_t *index_grid, const uint32_t *coords, int L, int B,
                                 uint4 *padded)
{
    const int slot = blockIdx.x, B1 = B + 1, nb = L / B;
    const uint32_t c = coords[slot];
    const int bx = c & 1023, by = (c >> 10) & 1023, bz = c >> 20;
    uint4 *dst = padded + (size_t)slot * B1 * B1 * B1;
    auto voxel = [&](int gx, int gy, int gz) {
        if (gx >= L || gy >= L || gz >= L) return make_uint2(0u, 0u);
        const int src = index_grid[((size_t)(gz / B) * nb + gy / B) * nb + gx / B];
        return src >= 0 ? atlas[(((size_t)src * B + gz % B) * B + gy % B) * B + gx % B] : make_uint2(0u, 0u);
    };
    for (int v = threadIdx.x; v < B1 * B1 * B1; v += blockDim.x) {
        const int lx = v % B1, ly = (v / B1) % B1, lz = v / (B1 * B1);
        const int gx = bx * B + lx, gy = by * B + ly, gz = bz * B + lz;
        dst[v] = merf::pair_bytes(voxel(gx, gy, gz), lx < B ? voxel(gx + 1, gy, gz) : make_uint2(0u, 0u));
    }
}

// Planes with a one-texel border that repeats their edge texels, [3][R+2][R+2] from [3][R][R],
// each stored as the texel pair (u, u + 1), bytes interleaved; the last column's upper texel is zero.
__global__ void border_planes_kernel(const uint2 *planes, int R, uint4 *bordered)
{
    const int Rp = R + 2;
    const size_t n = 3ull * Rp * Rp;
    auto texel = [&](int q, int u, int v) {
        const int su = min(max(u - 1, 0), R - 1), sv = min(max(v - 1, 0), R - 1);
        return planes[((size_t)q * R + sv) * R + su];
    };
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const int u = (int)(t % Rp), v = (int)((t / Rp) % Rp), q = (int)(t / ((size_t)Rp * Rp));
        bordered[t] = merf::pair_bytes(texel(q, u, v), u + 1 < Rp ? texel(q, u + 1, v) : make_uint2(0u, 0u));
    }
}

// Host side of the same layout: the 8 bytes of texel `src` as the lower texel of pair `lower`
// (even bytes) and, when given, the upper texel of pair `upper` (odd bytes).
static void put_in_pairs(const uint8_t *src, uint8_t *lower, uint8_t *upper)
{
    for (int k = 0; k < 8; ++k) {
        lower[2 * k] = src[k];
        if (upper) upper[2 * k + 1] = src[k];
    }
}

extern "C" {

merf_status merf_scene_upload(const merf_scene_desc *desc, const int32_t *index_grid, const uint8_t *atlas,
                              const uint8_t *planes, const uint8_t *const *occ_levels, const float *mlp_weights,
                              void *stream, merf_scene **out)
{
    const merf::NvtxRange nvtx_range("merf_scene_upload");
    merf_status st = check_desc(desc, MERF_STORAGE_U8_SPARSE);
    if (st) return st;
    if (!out) return fail(MERF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!index_grid || (desc->plane_res > 0 && !planes) || !mlp_weights || (desc->n_blocks > 0 && !atlas))
        return fail(MERF_ERR_INVALID_ARG, "a scene array is NULL");
    const size_t nb = (size_t)desc->grid_res / desc->block_size;
    for (size_t i = 0; i < nb * nb * nb; ++i)
        if (index_grid[i] < -1 || index_grid[i] >= desc->n_blocks)
            return fail(MERF_ERR_INVALID_ARG, "index_grid[%zu] = %d outside [-1, %d)", i, index_grid[i],
                        desc->n_blocks);
    if ((st = check_occupancy(desc, occ_levels))) return st;
    for (int i = 0; i < MERF_MLP_PARAMS; ++i)
        if (!std::isfinite(mlp_weights[i])) return fail(MERF_ERR_INVALID_ARG, "mlp_weights[%d] not finite", i);
    if (desc->n_blocks >= (1 << 24)) return fail(MERF_ERR_INVALID_ARG, "n_blocks %d >= 2^24", desc->n_blocks);
    // Device layout: each stored block gets a one-voxel apron copied from its +x/+y/+z
    // neighbours, and its index-grid entry carries in bits 24..30 a mask of the neighbours
    // (dx + 2 dy + 4 dz in 1..7, bit 23 + that number) that are not stored or lie past the
    // grid edge.
    const int B = desc->block_size, B1 = B + 1, L = desc->grid_res;
    const size_t R = desc->plane_res, nbi = nb;
    std::vector<uint8_t> apron;
    std::vector<int32_t> ig;
    try {
        apron.assign((size_t)desc->n_blocks * B1 * B1 * B1 * 16, 0);
        ig = index_with_neighbour_masks(index_grid, nbi);
    } catch (...) {
        return fail(MERF_ERR_OOM, "host memory for the padded atlas");
    }
    auto id_at = [&](size_t bx, size_t by, size_t bz) -> int32_t {
        if (bx >= nbi || by >= nbi || bz >= nbi) return -1;
        return index_grid[(bz * nbi + by) * nbi + bx];
    };
    for (size_t bz = 0; bz < nbi; ++bz)
        for (size_t by = 0; by < nbi; ++by)
            for (size_t bx = 0; bx < nbi; ++bx) {
                const int32_t id = id_at(bx, by, bz);
                if (id < 0) continue;
                uint8_t *dst = apron.data() + (size_t)id * B1 * B1 * B1 * 16;
                for (int lz = 0; lz < B1; ++lz)
                    for (int ly = 0; ly < B1; ++ly)
                        for (int lx = 0; lx < B1; ++lx) {
                            const size_t gx = bx * B + lx, gy = by * B + ly, gz = bz * B + lz;
                            if (gx >= (size_t)L || gy >= (size_t)L || gz >= (size_t)L) continue;
                            const int32_t src = id_at(gx / B, gy / B, gz / B);
                            if (src < 0) continue;
                            const uint8_t *sv = atlas + ((((size_t)src * B + gz % B) * B + gy % B) * B + gx % B) * 8;
                            uint8_t *pair = dst + (((size_t)lz * B1 + ly) * B1 + lx) * 16;
                            put_in_pairs(sv, pair, lx > 0 ? pair - 16 : nullptr);
                        }
            }
    // Each plane gets a one-texel border that repeats its edge texels, so that bilinear taps of
    // clamp-to-edge interpolation never need their coordinates clamped: [3][R+2][R+2].
    // (a grid-only scene, R = 0, has no planes at all)
    // Atlas voxels and plane texels are stored as pairs along x (the column axis), bytes
    // interleaved: the byte order the interpolation's dot products take.
    const size_t Rp = R + 2;
    std::vector<uint8_t> padded;
    try {
        padded.assign(R > 0 ? 3 * Rp * Rp * 16 : 0, 0);
    } catch (...) {
        return fail(MERF_ERR_OOM, "host memory for the bordered planes");
    }
    for (size_t q = 0; q < (R > 0 ? 3 : 0); ++q)
        for (size_t v = 0; v < Rp; ++v)
            for (size_t u = 0; u < Rp; ++u) {
                const size_t sv = v == 0 ? 0 : v > R ? R - 1 : v - 1, su = u == 0 ? 0 : u > R ? R - 1 : u - 1;
                uint8_t *pair = padded.data() + ((q * Rp + v) * Rp + u) * 16;
                put_in_pairs(planes + ((q * R + sv) * R + su) * 8, pair, u > 0 ? pair - 16 : nullptr);
            }
    return upload_common(desc, apron.data(), apron.size(), padded.data(), padded.size(), ig.data(),
                         nb * nb * nb * sizeof(int32_t), occ_levels, mlp_weights, stream, out);
}

merf_status merf_scene_upload_device(const merf_scene_desc *desc, const int32_t *d_index_grid,
                                     const uint8_t *d_atlas, const uint8_t *d_planes,
                                     const uint8_t *const *d_occ_levels, const float *d_mlp, void *stream,
                                     merf_scene **out)
{
    const merf::NvtxRange nvtx_range("merf_scene_upload_device");
    merf_status st = check_desc(desc, MERF_STORAGE_U8_SPARSE);
    if (st) return st;
    if (!out) return fail(MERF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!d_index_grid || (desc->plane_res > 0 && !d_planes) || !d_mlp || !d_occ_levels ||
        (desc->n_blocks > 0 && !d_atlas))
        return fail(MERF_ERR_INVALID_ARG, "a scene array is NULL");
    for (int l = 0; l < desc->n_occ_levels; ++l)
        if (!d_occ_levels[l]) return fail(MERF_ERR_INVALID_ARG, "occ_levels[%d] is NULL", l);
    if (desc->n_blocks >= (1 << 24)) return fail(MERF_ERR_INVALID_ARG, "n_blocks %d >= 2^24", desc->n_blocks);
    cudaStream_t cs = (cudaStream_t)stream;
    // the small arrays come to the host for the checks merf_scene_upload makes
    const size_t nb = (size_t)desc->grid_res / desc->block_size, n_index = nb * nb * nb;
    std::vector<int32_t> index(n_index);
    std::vector<std::vector<uint8_t>> occ(desc->n_occ_levels);
    std::vector<float> mlp(MERF_MLP_PARAMS);
    cudaError_t e = cudaMemcpyAsync(index.data(), d_index_grid, n_index * sizeof(int32_t), cudaMemcpyDeviceToHost, cs);
    for (int l = 0; l < desc->n_occ_levels && e == cudaSuccess; ++l) {
        occ[l].resize((size_t)desc->occ_res[l] * desc->occ_res[l] * desc->occ_res[l]);
        e = cudaMemcpyAsync(occ[l].data(), d_occ_levels[l], occ[l].size(), cudaMemcpyDeviceToHost, cs);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(mlp.data(), d_mlp, sizeof(float) * MERF_MLP_PARAMS, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return fail(MERF_ERR_CUDA, "reading the scene's index, occupancy and MLP: %s", cudaGetErrorString(e));
    std::vector<uint32_t> coords((size_t)std::max(desc->n_blocks, 1), 0xffffffffu);
    for (size_t i = 0; i < n_index; ++i) {
        if (index[i] < -1 || index[i] >= desc->n_blocks)
            return fail(MERF_ERR_INVALID_ARG, "index_grid[%zu] = %d outside [-1, %d)", i, index[i], desc->n_blocks);
        if (index[i] >= 0) {
            if (coords[index[i]] != 0xffffffffu)
                return fail(MERF_ERR_INVALID_ARG, "atlas slot %d is named by two index-grid entries", index[i]);
            coords[index[i]] = (uint32_t)(i % nb) | ((uint32_t)((i / nb) % nb) << 10) | ((uint32_t)(i / (nb * nb)) << 20);
        }
    }
    for (int b = 0; b < desc->n_blocks; ++b)
        if (coords[b] == 0xffffffffu) return fail(MERF_ERR_INVALID_ARG, "atlas slot %d is named by no index-grid entry", b);
    std::vector<const uint8_t *> occ_ptrs(desc->n_occ_levels);
    for (int l = 0; l < desc->n_occ_levels; ++l) occ_ptrs[l] = occ[l].data();
    if ((st = check_occupancy(desc, occ_ptrs.data()))) return st;
    for (int i = 0; i < MERF_MLP_PARAMS; ++i)
        if (!std::isfinite(mlp[i])) return fail(MERF_ERR_INVALID_ARG, "mlp_weights[%d] not finite", i);
    std::vector<int32_t> ig;
    try {
        ig = index_with_neighbour_masks(index.data(), nb);
    } catch (...) {
        return fail(MERF_ERR_OOM, "host memory for the index grid");
    }
    // Device layout as merf_scene_upload builds it, made on the device: the padded atlas and the
    // bordered planes by kernels from the caller's arrays; the rest copied.
    const int B = desc->block_size, B1 = B + 1;
    const size_t R = desc->plane_res, Rp = R + 2;
    const size_t atlas_bytes = (size_t)desc->n_blocks * B1 * B1 * B1 * 16, plane_bytes = R > 0 ? 3 * Rp * Rp * 16 : 0;
    size_t total = atlas_bytes + plane_bytes + n_index * sizeof(int32_t) + merf::kMlpBlockBytes;
    for (int l = 0; l < desc->n_occ_levels; ++l) total += occ[l].size();
    if (g_budget && total > g_budget)
        return fail(MERF_ERR_OOM, "scene needs %zu device bytes, budget is %zu", total, g_budget);
    merf_scene *sc = new merf_scene();
    sc->desc = *desc;
    cudaGetDevice(&sc->device);
    uint32_t *d_coords = nullptr;
    auto bail = [&](merf_status code, const char *what, cudaError_t err) {
        cudaGetLastError();
        cudaFree(d_coords);
        free_scene_memory(sc);
        delete sc;
        return fail(code, "%s: %s", what, cudaGetErrorString(err));
    };
    struct Item { void **dst; size_t n; };
    std::vector<Item> items = {{&sc->atlas, atlas_bytes}, {&sc->planes, plane_bytes},
                               {&sc->index_grid, n_index * sizeof(int32_t)}, {&sc->mlp, merf::kMlpBlockBytes},
                               {(void **)&d_coords, coords.size() * sizeof(uint32_t)}};
    for (int l = 0; l < desc->n_occ_levels; ++l) items.push_back({&sc->occ[l], occ[l].size()});
    for (auto &it : items) {
        if (it.n == 0) continue;
        if ((e = cudaMalloc(it.dst, it.n)) != cudaSuccess)
            return bail(e == cudaErrorMemoryAllocation ? MERF_ERR_OOM : MERF_ERR_CUDA, "cudaMalloc", e);
    }
    e = cudaMemcpyAsync(sc->index_grid, ig.data(), n_index * sizeof(int32_t), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_coords, coords.data(), coords.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, cs);
    for (int l = 0; l < desc->n_occ_levels && e == cudaSuccess; ++l)
        e = cudaMemcpyAsync(sc->occ[l], d_occ_levels[l], occ[l].size(), cudaMemcpyDeviceToDevice, cs);
    if (e == cudaSuccess) e = put_mlp_block(sc->mlp, d_mlp, cudaMemcpyDeviceToDevice, cs);
    if (e == cudaSuccess && desc->n_blocks > 0) {
        pad_atlas_kernel<<<desc->n_blocks, 256, 0, cs>>>((const uint2 *)d_atlas, d_index_grid, d_coords, desc->grid_res,
                                                         B, (uint4 *)sc->atlas);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && R > 0) {
        border_planes_kernel<<<4 * 148, 256, 0, cs>>>((const uint2 *)d_planes, (int)R, (uint4 *)sc->planes);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return bail(MERF_ERR_CUDA, "building the scene on the device", e);
    cudaFree(d_coords);
    sc->bytes = total;
    *out = sc;
    return ok();
}

merf_status merf_scene_upload_dense(const merf_scene_desc *desc, const float *grid, const float *planes,
                                    const uint8_t *const *occ_levels, const float *mlp_weights, void *stream,
                                    merf_scene **out)
{
    const merf::NvtxRange nvtx_range("merf_scene_upload_dense");
    merf_status st = check_desc(desc, MERF_STORAGE_F32_DENSE);
    if (st) return st;
    if (!out) return fail(MERF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!grid || !planes || !mlp_weights) return fail(MERF_ERR_INVALID_ARG, "a scene array is NULL");
    if ((st = check_occupancy(desc, occ_levels))) return st;
    const size_t L = desc->grid_res, R = desc->plane_res;
    return upload_common(desc, grid, L * L * L * 8 * sizeof(float), planes, 3 * R * R * 8 * sizeof(float),
                         nullptr, 0, occ_levels, mlp_weights, stream, out);
}

}  // extern "C"

namespace {

static_assert(sizeof(merf_scene_file_header) == 256, "scene file header is 256 bytes");

// Byte offsets of a scene file's arrays (the header first, each array 64-byte aligned).
struct SceneFileLayout {
    size_t grid = 0, grid_bytes = 0;       // index grid (uint8 storage) or float grid
    size_t atlas = 0, atlas_bytes = 0;     // uint8 storage only
    size_t planes = 0, plane_bytes = 0;    // none for a grid-only scene
    size_t occ[MERF_MAX_OCC_LEVELS] = {};
    size_t mlp = 0, end = 0;
};

// desc has passed check_desc and n_blocks <= (L/B)^3, so no size below overflows.
SceneFileLayout scene_file_layout(const merf_scene_desc &d)
{
    SceneFileLayout f;
    size_t at = sizeof(merf_scene_file_header);
    auto place = [&at](size_t &off, size_t n) {
        off = (at + 63) & ~(size_t)63;
        at = off + n;
    };
    const size_t L = d.grid_res, R = d.plane_res;
    if (d.storage == MERF_STORAGE_U8_SPARSE) {
        const size_t B = d.block_size, nb = L / B;
        f.grid_bytes = nb * nb * nb * sizeof(int32_t);
        place(f.grid, f.grid_bytes);
        f.atlas_bytes = (size_t)d.n_blocks * B * B * B * MERF_CHANNELS;
        place(f.atlas, f.atlas_bytes);
        f.plane_bytes = 3 * R * R * MERF_CHANNELS;
    } else {
        f.grid_bytes = L * L * L * MERF_CHANNELS * sizeof(float);
        place(f.grid, f.grid_bytes);
        f.plane_bytes = 3 * R * R * MERF_CHANNELS * sizeof(float);
    }
    if (f.plane_bytes) place(f.planes, f.plane_bytes);
    for (int l = 0; l < d.n_occ_levels; ++l) {
        const size_t n = d.occ_res[l];
        place(f.occ[l], n * n * n);
    }
    place(f.mlp, sizeof(float) * MERF_MLP_PARAMS);
    f.end = at;
    return f;
}

struct Mapping {
    void *p = MAP_FAILED;
    size_t n = 0;
    ~Mapping()
    {
        if (p != MAP_FAILED) munmap(p, n);
    }
};

}  // namespace

extern "C" {

merf_status merf_scene_load(const char *path, void *stream, merf_scene **out)
{
    const merf::NvtxRange nvtx_range("merf_scene_load");
    if (!out) return fail(MERF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!path) return fail(MERF_ERR_INVALID_ARG, "path is NULL");
    const int fd = open(path, O_RDONLY | O_CLOEXEC);
    if (fd < 0) return fail(MERF_ERR_INVALID_ARG, "cannot open %s: %s", path, strerror(errno));
    struct stat sb;
    if (fstat(fd, &sb) != 0 || sb.st_size < (off_t)sizeof(merf_scene_file_header)) {
        close(fd);
        return fail(MERF_ERR_INVALID_ARG, "%s is shorter than a scene file header", path);
    }
    Mapping m;
    m.n = (size_t)sb.st_size;
    m.p = mmap(nullptr, m.n, PROT_READ, MAP_PRIVATE, fd, 0);
    close(fd);
    if (m.p == MAP_FAILED) return fail(MERF_ERR_INVALID_ARG, "cannot map %s: %s", path, strerror(errno));
    merf_scene_file_header h;
    memcpy(&h, m.p, sizeof h);
    if (memcmp(h.magic, "MERFSCN1", 8) != 0) return fail(MERF_ERR_INVALID_ARG, "%s is not a MERF scene file", path);
    if (h.version != 1 || h.header_bytes != sizeof h)
        return fail(MERF_ERR_INVALID_ARG, "%s: version %u with a %u-byte header (1 and 256 expected)", path,
                    h.version, h.header_bytes);
    if (h.desc.storage != MERF_STORAGE_U8_SPARSE && h.desc.storage != MERF_STORAGE_F32_DENSE)
        return fail(MERF_ERR_INVALID_ARG, "%s: storage %d", path, h.desc.storage);
    merf_status st = check_desc(&h.desc, h.desc.storage);
    if (st) return st;
    if (h.desc.storage == MERF_STORAGE_U8_SPARSE) {
        const long long nb = h.desc.grid_res / h.desc.block_size;
        if (h.desc.n_blocks > nb * nb * nb)
            return fail(MERF_ERR_INVALID_ARG, "%s: %d blocks for an index grid of %lld", path, h.desc.n_blocks,
                        nb * nb * nb);
    }
    const SceneFileLayout f = scene_file_layout(h.desc);
    if (h.file_bytes != m.n || f.end != m.n)
        return fail(MERF_ERR_INVALID_ARG, "%s holds %zu bytes; its header says %llu and its descriptor needs %zu",
                    path, m.n, (unsigned long long)h.file_bytes, f.end);
    const uint8_t *base = (const uint8_t *)m.p;
    const uint8_t *occ[MERF_MAX_OCC_LEVELS] = {};
    for (int l = 0; l < h.desc.n_occ_levels; ++l) occ[l] = base + f.occ[l];
    const float *mlp = (const float *)(base + f.mlp);
    if (h.desc.storage == MERF_STORAGE_U8_SPARSE)
        return merf_scene_upload(&h.desc, (const int32_t *)(base + f.grid), base + f.atlas,
                                 f.plane_bytes ? base + f.planes : nullptr, occ, mlp, stream, out);
    return merf_scene_upload_dense(&h.desc, (const float *)(base + f.grid), (const float *)(base + f.planes), occ,
                                   mlp, stream, out);
}

void merf_scene_free(merf_scene *scene)
{
    if (!scene) return;
    cudaDeviceSynchronize();
    free_scene_memory(scene);
    delete scene;
}

size_t merf_scene_device_bytes(const merf_scene *scene) { return scene ? scene->bytes : 0; }

merf_status merf_render_aux(const merf_scene *scene, const merf_camera *cams, int n_cams, int W, int H, float *out,
                            float *aux, unsigned long long *counters, const merf_render_opts *opts, void *stream)
{
    const merf::NvtxRange nvtx_range("merf_render");
    merf_status st = check_frame(scene, cams, n_cams, W, H);
    if (st) return st;
    if ((st = check_opts(opts))) return st;
    if (!out) return fail(MERF_ERR_INVALID_ARG, "out is NULL");
    return launch_render(scene, cams, n_cams, W, H, out, aux, counters, opts, (cudaStream_t)stream);
}

merf_status merf_render(const merf_scene *scene, const merf_camera *cams, int n_cams, int W, int H, float *out,
                        const merf_render_opts *opts, void *stream)
{
    return merf_render_aux(scene, cams, n_cams, W, H, out, nullptr, nullptr, opts, stream);
}

namespace {
// Per-device copy stream and events of merf_render_host (created on first use, kept until exit).
struct HostCopy {
    cudaStream_t stream = nullptr;
    std::vector<cudaEvent_t> events;
};
std::mutex g_host_copy_mu;
HostCopy g_host_copy[64];
}  // namespace

merf_status merf_render_host(const merf_scene *scene, const merf_camera *cams, int n_cams, int W, int H,
                             float *d_staging, float *h_out, const merf_render_opts *opts, void *stream)
{
    const merf::NvtxRange nvtx_range("merf_render_host");
    if (!h_out) return fail(MERF_ERR_INVALID_ARG, "h_out is NULL");
    merf_status st = check_frame(scene, cams, n_cams, W, H);
    if (st) return st;
    if ((st = check_opts(opts))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // Page-locked host memory that the device can address (cudaHostAlloc, or registered with
    // cudaHostRegister, under unified addressing): the kernel stores the image there directly,
    // one launch for all cameras, no staging buffer and no copy.
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, h_out) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer) {
        if ((st = launch_render(scene, cams, n_cams, W, H, (float *)pa.devicePointer, nullptr, nullptr, opts, s)))
            return st;
        const cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(MERF_ERR_CUDA, "render_host: %s", cudaGetErrorString(e));
        return ok();
    }
    cudaGetLastError();   // a pageable pointer is not an error here
    if (!d_staging) return fail(MERF_ERR_INVALID_ARG, "d_staging is NULL and h_out is not page-locked");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return fail(MERF_ERR_UNSUPPORTED, "device ordinal %d", dev);
    const size_t per = (size_t)W * H * 3;
    std::lock_guard<std::mutex> lk(g_host_copy_mu);
    HostCopy &hc = g_host_copy[dev];
    cudaError_t e = cudaSuccess;
    if (!hc.stream) e = cudaStreamCreateWithFlags(&hc.stream, cudaStreamNonBlocking);
    while (e == cudaSuccess && (int)hc.events.size() < n_cams) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) hc.events.push_back(ev);
    }
    if (e != cudaSuccess) return fail(MERF_ERR_CUDA, "render_host resources: %s", cudaGetErrorString(e));
    // Otherwise camera c renders on the caller's stream into d_staging while camera c-1's image
    // is copied to the host on a second stream, so the copies hide behind the rendering.
    for (int c = 0; c < n_cams; ++c) {
        if ((st = launch_render(scene, cams + c, 1, W, H, d_staging + c * per, nullptr, nullptr, opts, s))) return st;
        e = cudaEventRecord(hc.events[c], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(hc.stream, hc.events[c], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_out + c * per, d_staging + c * per, per * sizeof(float), cudaMemcpyDeviceToHost,
                                hc.stream);
        if (e != cudaSuccess) return fail(MERF_ERR_CUDA, "render_host: %s", cudaGetErrorString(e));
    }
    e = cudaStreamSynchronize(hc.stream);
    if (e != cudaSuccess) return fail(MERF_ERR_CUDA, "render_host copy: %s", cudaGetErrorString(e));
    return ok();
}

// Staging area of merf_render_host_noalloc: device memory that belongs to the library, so a
// caller that cannot allocate can still render into host memory.  Host code must not use the
// name as a pointer (it denotes a host-side shadow); the device address is looked up once per
// device with cudaGetSymbolAddress.
static __device__ __align__(256) float g_noalloc_staging[MERF_NOALLOC_STAGING_BYTES / sizeof(float)];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
float *g_noalloc_ptr[kMaxDevices] = {};
}  // namespace

merf_status merf_trace(const merf_scene *scene, const merf_camera *cams, int n_cams, int W, int H, uint32_t *mask,
                       int words, int32_t *n_lattice, const merf_render_opts *opts, void *stream)
{
    const merf::NvtxRange nvtx_range("merf_trace");
    merf_status st = check_frame(scene, cams, n_cams, W, H);
    if (st) return st;
    if ((st = check_opts(opts))) return st;
    if (!mask || !n_lattice) return fail(MERF_ERR_INVALID_ARG, "mask / n_lattice is NULL");
    if (words < 1 || words > 4096) return fail(MERF_ERR_INVALID_ARG, "words %d not in [1, 4096]", words);
    merf::RenderParams P = make_params(scene, opts, W, H);
    P.mask = mask;
    P.nlat = n_lattice;
    P.words = words;
    cudaStream_t s = (cudaStream_t)stream;
    for (int c0 = 0; c0 < n_cams; c0 += merf::kMaxCams) {
        const int nc = std::min(merf::kMaxCams, n_cams - c0);
        P.cam0 = c0;
        for (int c = 0; c < nc; ++c) memcpy(P.cams.m[c], &cams[c0 + c], sizeof(merf_camera));
        const dim3 grid((W + merf::kTileW - 1) / merf::kTileW, (H + merf::kTileH - 1) / merf::kTileH, nc);
        merf::trace_kernel<<<grid, merf::kThreads, 0, s>>>(P);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(MERF_ERR_CUDA, "trace launch: %s", cudaGetErrorString(e));
    }
    return ok();
}

merf_status merf_render_host_noalloc(const merf_scene *scene, const merf_camera *cams, int n_cams, int W, int H,
                                     float *h_out, const merf_render_opts *opts, void *stream)
{
    const merf::NvtxRange nvtx_range("merf_render_host_noalloc");
    if (!h_out) return fail(MERF_ERR_INVALID_ARG, "h_out is NULL");
    merf_status st = check_frame(scene, cams, n_cams, W, H);
    if (st) return st;
    if ((st = check_opts(opts))) return st;
    const size_t bytes = (size_t)n_cams * W * H * 3 * sizeof(float);
    if (bytes > (size_t)MERF_NOALLOC_STAGING_BYTES)
        return fail(MERF_ERR_INVALID_ARG,
                    "image of %zu bytes exceeds the %d-byte staging area of merf_render_host_noalloc "
                    "(render fewer cameras per call or use merf_render_host)",
                    bytes, (int)MERF_NOALLOC_STAGING_BYTES);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(MERF_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(MERF_ERR_UNSUPPORTED, "device ordinal %d >= %d", dev, kMaxDevices);
    float *staging = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_staging);
            if (e != cudaSuccess || !p)
                return fail(MERF_ERR_CUDA, "cudaGetSymbolAddress(staging): %s", cudaGetErrorString(e));
            g_noalloc_ptr[dev] = (float *)p;
        }
        staging = g_noalloc_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = launch_render(scene, cams, n_cams, W, H, staging, nullptr, nullptr, opts, s))) return st;
    e = cudaMemcpyAsync(h_out, staging, bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(MERF_ERR_CUDA, "render_host_noalloc copy: %s", cudaGetErrorString(e));
    return ok();
}

merf_status merf_scene_set_dense(merf_scene *scene, const float *d_grid, const float *d_planes, const float *d_mlp,
                                 void *stream)
{
    if (!scene || !d_grid || !d_planes || !d_mlp) return fail(MERF_ERR_INVALID_ARG, "NULL argument");
    if (scene->desc.storage != MERF_STORAGE_F32_DENSE)
        return fail(MERF_ERR_UNSUPPORTED, "merf_scene_set_dense needs a dense float scene");
    const size_t L = scene->desc.grid_res, R = scene->desc.plane_res;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(scene->atlas, d_grid, L * L * L * 8 * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(scene->planes, d_planes, 3 * R * R * 8 * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = put_mlp_block(scene->mlp, d_mlp, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return fail(MERF_ERR_CUDA, "set_dense: %s", cudaGetErrorString(e));
    ++scene->param_version;
    return ok();
}

unsigned long long merf_scene_param_version(const merf_scene *scene)
{
    return scene ? scene->param_version : 0ull;
}

merf_status merf_render_backward(const merf_scene *scene, const merf_camera *cams, int n_cams, int W, int H,
                                 const float *d_out, float *g_grid, float *g_planes, float *g_mlp,
                                 const merf_render_opts *opts, void *stream)
{
    return merf_render_backward_aux(scene, cams, n_cams, W, H, d_out, nullptr, g_grid, g_planes, g_mlp, opts,
                                    stream);
}

merf_status merf_render_backward_aux(const merf_scene *scene, const merf_camera *cams, int n_cams, int W, int H,
                                     const float *d_out, const float *aux, float *g_grid, float *g_planes,
                                     float *g_mlp, const merf_render_opts *opts, void *stream)
{
    const merf::NvtxRange nvtx_range("merf_render_backward");
    merf_status st = check_frame(scene, cams, n_cams, W, H);
    if (st) return st;
    if ((st = check_opts(opts))) return st;
    if (!d_out || !g_grid || !g_planes || !g_mlp) return fail(MERF_ERR_INVALID_ARG, "NULL gradient buffer");
    if (scene->desc.storage != MERF_STORAGE_F32_DENSE)
        return fail(MERF_ERR_UNSUPPORTED, "the adjoint is defined for dense float scenes");
    if (opts->precision != MERF_PREC_FP32) return fail(MERF_ERR_UNSUPPORTED, "the adjoint runs in FP32");
    if (opts->contraction != 0) return fail(MERF_ERR_UNSUPPORTED, "the adjoint follows contract_pi only");
    merf::RenderParams R = make_params(scene, opts, W, H);
    merf::BackwardParams P;
    memset(&P, 0, sizeof P);
    P.fv = R.fv;
    P.occ = R.occ;
    P.mlp = R.mlp;
    P.d_out = d_out;
    P.aux = aux;
    P.g_grid = g_grid;
    P.g_planes = g_planes;
    P.g_mlp = g_mlp;
    P.W = W;
    P.H = H;
    P.step = opts->step;
    P.t_term = opts->t_term;
    P.early_term = opts->early_term;
    cudaStream_t s = (cudaStream_t)stream;
    for (int c0 = 0; c0 < n_cams; c0 += merf::kMaxCams) {
        const int nc = std::min(merf::kMaxCams, n_cams - c0);
        P.cam0 = c0;
        for (int c = 0; c < nc; ++c) memcpy(P.cams.m[c], &cams[c0 + c], sizeof(merf_camera));
        const dim3 grid((W + merf::kTileW - 1) / merf::kTileW, (H + merf::kTileH - 1) / merf::kTileH, nc);
        if (merf::gather_geometry(scene->desc) == merf::kGeoDense32)
            merf::backward_kernel<merf::kGeoDense32><<<grid, merf::kThreads, 0, s>>>(P);
        else
            merf::backward_kernel<merf::kGeoRuntime><<<grid, merf::kThreads, 0, s>>>(P);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(MERF_ERR_CUDA, "backward launch: %s", cudaGetErrorString(e));
    }
    return ok();
}

void merf_set_device_budget(size_t bytes) { g_budget = bytes; }

const char *merf_last_error(void) { return g_err.c_str(); }

#ifdef MERF_DEBUG_BOUNDS
const char *merf_version(void) { return "merf-b300 0.1 (sm_103a, bounds-checked build)"; }
#else
const char *merf_version(void) { return "merf-b300 0.1 (sm_103a)"; }
#endif

merf_status merf_check_device(void *stream, int self_test)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (self_test < 0 || self_test > 2) return fail(MERF_ERR_INVALID_ARG, "self_test %d not in 0..2", self_test);
    if (self_test == 2) {
        wait_timeout_self_test_kernel<<<1, 1, 0, s>>>();
        if (cudaGetLastError() != cudaSuccess) return fail(MERF_ERR_CUDA, "self-test launch failed");
    }
#ifdef MERF_DEBUG_BOUNDS
    if (self_test == 1) {
        status_self_test_kernel<<<1, 1, 0, s>>>();
        if (cudaGetLastError() != cudaSuccess) return fail(MERF_ERR_CUDA, "self-test launch failed");
    }
#else
    if (self_test == 1) return fail(MERF_ERR_UNSUPPORTED, "the bounds self-test needs the bounds-checked build");
#endif
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(MERF_ERR_CUDA, "check_device: %s", cudaGetErrorString(e));
    unsigned int word = 0, zero = 0;
    e = cudaMemcpyFromSymbol(&word, merf::g_status, sizeof word);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(merf::g_status, &zero, sizeof zero);
    if (e != cudaSuccess) return fail(MERF_ERR_CUDA, "check_device: %s", cudaGetErrorString(e));
    word |= merf::take_server_status();
    const unsigned bounds = merf::kBadIndexGrid | merf::kBadAtlas | merf::kBadPlane | merf::kBadOcc | merf::kBadDense |
                            merf::kStatusSelfTest;
    if (word & bounds)
        return fail(MERF_ERR_DEVICE_BOUNDS, "device status 0x%08x:%s%s%s%s%s%s%s", word,
                    (word & merf::kBadIndexGrid) ? " index-grid" : "", (word & merf::kBadAtlas) ? " atlas" : "",
                    (word & merf::kBadPlane) ? " plane" : "", (word & merf::kBadOcc) ? " occupancy" : "",
                    (word & merf::kBadDense) ? " dense" : "", (word & merf::kWaitTimeout) ? " wait-timeout" : "",
                    (word & merf::kStatusSelfTest) ? " self-test" : "");
    if (word & merf::kWaitTimeout)
        return fail(MERF_ERR_TIMEOUT, "device status 0x%08x: a tensor-core completion wait gave up", word);
    return ok();
}

}  // extern "C"
