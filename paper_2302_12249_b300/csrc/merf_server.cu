// merf_server.cu -- the serving form's device side (declared in merf.h): the persistent tile
// kernel, and the CUDA backend through which the scheduler of serve_sched.h (admission by pool
// memory, continuous batching, completion, cancellation) runs it.
//
// An iteration is one launch of a captured CUDA graph: work-list upload, counter reset and
// serve_kernel.  The kernel keeps one CTA per resident slot (SMs x CTAs per SM) and pulls tiles
// from the work list with an atomic counter, so long and short requests balance across SMs.  Each
// CTA renders its tile with the same march and deferred MLP as render_kernel; the MLP weights in
// shared memory are fetched again (one bulk copy) when a tile belongs to another scene.  The only
// device-side waits are the CTA's own bounded waits on its copies and MMAs.
// The scheduler's two iteration slots are two work buffers and two graphs on one compute stream;
// a finished request's image is copied to host memory on a second stream, and the copy's event
// completes the request.
#include <cuda_runtime.h>

#include <cstring>

#include "merf.h"
#include "nvtx.h"
#include "render.cuh"
#include "scene.h"
#include "serve_sched.h"

namespace merf {

static_assert(kServeTileW == kTileW && kServeTileH == kTileH, "a serving tile is one render CTA");
static_assert(kServeMaxTiles <= (1 << 20) && kServeMaxReq <= (1 << 12), "tile code: request << 20 | tile");

struct ServeScene {
    FieldView fv;
    OccView occ;
    const float *mlp;
};

struct ServeParams {
    ServeScene scenes[kServeMaxScenes];
    const ServeWork *work;
    int *counter;
    float *pool;
    float step, t_term;
    int early_term;
};

template <int kPrec, int kGeo>
__global__ void __launch_bounds__(kThreads, (kMinBlocks<0, kPrec>)) serve_kernel(const __grid_constant__ ServeParams P)
{
    __shared__ MlpSmem<kPrec> ms;
    __shared__ int s_tile;
    ms.init();                          // the first barrier below publishes it
    const int n_tiles = P.work->n_tiles;
    int cur_scene = -1;
    UmmaState us;
    uint32_t wphase = 0, lost = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(P.counter, 1);
        __syncthreads();
        const int tile = s_tile;
        if (tile >= n_tiles) break;
        const uint32_t code = P.work->tiles[tile];
        const ServeReq &R = P.work->req[code >> 20];
        const int sc = R.scene;
        // Uniform across the CTA.  The barriers since the last tile's MLP ordered every read of
        // the old weights before this copy.
        const bool fetched = sc != cur_scene;
        if (fetched) {
            ms.fetch(P.scenes[sc].mlp);     // lands while the rays march
            cur_scene = sc;
        }
        const int tl = (int)(code & 0xfffffu);
        const int tx = tl % R.tiles_x, ty = tl / R.tiles_x;
        const int i = tx * kTileW + (warp & 1) * 8 + (lane & 7);
        const int j = ty * kTileH + (warp >> 1) * 4 + (lane >> 3);
        const bool inside = (i < R.W) && (j < R.H);
        RayState r;
        ray_state_init(r);
        if (inside)
            march_ray<0, kPrec, kGeo>(P.scenes[sc].fv, P.scenes[sc].occ, R.cam, i, j, P.step, P.t_term, P.early_term, r);
        float h[3];
        // A copy or an MMA round that did not complete ends this CTA's work: no further copy or
        // MMA is issued, the tile is left unwritten, and the status word reports it.
        if (fetched && !__syncthreads_and(ms.wait(wphase, lost))) break;
        deferred_mlp<kPrec>(ms, us, r, inside, h);
        if (!__syncthreads_and(us.ok)) break;
        if (inside) {
            float *o = P.pool + R.out_off + ((size_t)j * R.W + i) * 3;
            o[0] = r.cd[0] + h[0];
            o[1] = r.cd[1] + h[1];
            o[2] = r.cd[2] + h[2];
        }
        __syncthreads();                // s_tile and the weights are reused next iteration
    }
    ms.fini(us, lost);
}

unsigned int take_server_status()
{
    unsigned int word = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&word, g_status, sizeof word) != cudaSuccess) return 0;
    cudaMemcpyToSymbol(g_status, &zero, sizeof zero);
    return word;
}

// The device behind the scheduler: iteration slot b is work buffer b and captured graph b on the
// compute stream; images leave the pool on the copy stream, one event per request.
class CudaServeBackend final : public ServeBackend {
public:
    int device = 0, grid = 0;
    ServeParams params[2];
    float *d_pool = nullptr;
    ServeWork *h_work[2] = {nullptr, nullptr}, *d_work[2] = {nullptr, nullptr};
    int *d_counter = nullptr;
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaStream_t s_comp = nullptr, s_copy = nullptr;
    cudaEvent_t ev_iter[2] = {nullptr, nullptr};

    ~CudaServeBackend() override
    {
        drain();
        for (int b = 0; b < 2; ++b) {
            if (exec[b]) cudaGraphExecDestroy(exec[b]);
            if (graph[b]) cudaGraphDestroy(graph[b]);
            if (ev_iter[b]) cudaEventDestroy(ev_iter[b]);
            if (h_work[b]) cudaFreeHost(h_work[b]);
            if (d_work[b]) cudaFree(d_work[b]);
        }
        if (d_counter) cudaFree(d_counter);
        if (d_pool) cudaFree(d_pool);
        if (s_comp) cudaStreamDestroy(s_comp);
        if (s_copy) cudaStreamDestroy(s_copy);
    }

    void thread_init() override { cudaSetDevice(device); }
    ServeWork *work(int b) override { return h_work[b]; }

    bool launch(int b) override
    {
        const NvtxRange nvtx_range("merf_server_iteration");
        return cudaGraphLaunch(exec[b], s_comp) == cudaSuccess && cudaEventRecord(ev_iter[b], s_comp) == cudaSuccess;
    }

    int poll_iter(int b) override { return poll(ev_iter[b]); }

    merf_status req_init(ServeRequest &r) override
    {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return MERF_ERR_CUDA;
        r.dev = e;
        return MERF_OK;
    }

    void req_free(ServeRequest &r) override
    {
        if (r.dev) cudaEventDestroy((cudaEvent_t)r.dev);
        r.dev = nullptr;
    }

    bool copy_out(ServeRequest &r) override
    {
        const NvtxRange nvtx_range("merf_server_copy_out");
        return cudaMemcpyAsync(r.h_out, d_pool + r.pool_off, r.floats * sizeof(float), cudaMemcpyDeviceToHost,
                               s_copy) == cudaSuccess &&
               cudaEventRecord((cudaEvent_t)r.dev, s_copy) == cudaSuccess;
    }

    int poll_copy(ServeRequest &r) override { return poll((cudaEvent_t)r.dev); }

    void drain() override
    {
        if (s_comp) cudaStreamSynchronize(s_comp);
        if (s_copy) cudaStreamSynchronize(s_copy);
    }

private:
    static int poll(cudaEvent_t e)
    {
        const cudaError_t q = cudaEventQuery(e);
        return q == cudaErrorNotReady ? 0 : q == cudaSuccess ? 1 : -1;
    }
};

}  // namespace merf

struct merf_server {
    merf::CudaServeBackend *be = nullptr;
    merf::ServeScheduler *sched = nullptr;
};

namespace {

merf_status serve_err(merf_status s, const char *msg)
{
    return s == MERF_OK ? merf::clear_error() : merf::set_error(s, "%s", msg);
}

template <int kPrec, int kGeo>
merf_status capture(merf::CudaServeBackend *s, int b)
{
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
        return merf::set_error(MERF_ERR_CUDA, "server: stream creation failed");
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_work[b], s->h_work[b], sizeof(merf::ServeWork), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_counter + b, 0, sizeof(int), cs);
    if (e == cudaSuccess) {
        merf::serve_kernel<kPrec, kGeo><<<s->grid, merf::kThreads, 0, cs>>>(s->params[b]);
        e = cudaGetLastError();
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&s->exec[b], g, 0);
    s->graph[b] = g;
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return merf::set_error(MERF_ERR_CUDA, "server graph capture: %s", cudaGetErrorString(e));
    return MERF_OK;
}

// One CTA per resident slot.  The launch bounds reserve registers for kMinBlocks CTAs per SM and
// their shared memory and tensor memory (32 columns each) fit beside one another, but the
// occupancy query answers 1 for the FP16/BF16 kernels, which allocate tensor memory at run time
// (measured: 148 CTAs on 148 SMs and 2.8x less serving throughput), so the larger of the two is
// taken.  The CTAs never wait for one another, so a slot that is not resident only starts late.
template <int kPrec, int kGeo>
int resident_grid()
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, merf::serve_kernel<kPrec, kGeo>, merf::kThreads, 0) !=
        cudaSuccess) {
        cudaGetLastError();
        per = 0;
    }
    return std::max(1, sms) * std::max(per, merf::kMinBlocks<0, kPrec>);
}

}  // namespace

extern "C" {

merf_status merf_server_create(const merf_scene *const *scenes, int n_scenes, const merf_server_opts *opts,
                               merf_server **out)
{
    if (!out) return merf::set_error(MERF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!scenes || n_scenes < 1 || n_scenes > merf::kServeMaxScenes)
        return merf::set_error(MERF_ERR_INVALID_ARG, "n_scenes %d not in [1, %d]", n_scenes, merf::kServeMaxScenes);
    if (!opts) return merf::set_error(MERF_ERR_INVALID_ARG, "opts is NULL");
    if (opts->max_tiles_per_iter < 1 || opts->max_tiles_per_iter > merf::kServeMaxTiles)
        return merf::set_error(MERF_ERR_INVALID_ARG, "max_tiles_per_iter %d not in [1, %d]", opts->max_tiles_per_iter,
                               merf::kServeMaxTiles);
    if (opts->max_tiles_backlog != 0 &&
        (opts->max_tiles_backlog < opts->max_tiles_per_iter || opts->max_tiles_backlog > merf::kServeMaxTiles))
        return merf::set_error(MERF_ERR_INVALID_ARG, "max_tiles_backlog %d: 0 or in [max_tiles_per_iter, %d]",
                               opts->max_tiles_backlog, merf::kServeMaxTiles);
    if (opts->precision != MERF_PREC_FP32 && opts->precision != MERF_PREC_FP16 && opts->precision != MERF_PREC_BF16)
        return merf::set_error(MERF_ERR_INVALID_ARG, "precision %d is not a MERF_PREC_* value", opts->precision);
    if (!(opts->step >= 1e-5f) || !(opts->step < 1e30f) || !(opts->t_term >= 0.0f) || !(opts->t_term < 1.0f) ||
        (opts->early_term != 0 && opts->early_term != 1))
        return merf::set_error(MERF_ERR_INVALID_ARG, "step / t_term / early_term invalid");
    if (opts->pool_bytes < 64 * sizeof(float))
        return merf::set_error(MERF_ERR_INVALID_ARG, "pool_bytes %zu too small", opts->pool_bytes);
    for (int k = 0; k < n_scenes; ++k) {
        if (!scenes[k]) return merf::set_error(MERF_ERR_INVALID_ARG, "scene %d is NULL", k);
        if (scenes[k]->desc.storage != MERF_STORAGE_U8_SPARSE || scenes[k]->desc.plane_res == 0)
            return merf::set_error(MERF_ERR_UNSUPPORTED,
                                   "scene %d: the server renders uint8 block-sparse scenes with planes", k);
    }
    merf::CudaServeBackend *s = new merf::CudaServeBackend();
    cudaGetDevice(&s->device);
    const int prec = opts->precision;
    // one persistent kernel serves every scene: the paper-geometry gather only if all have it
    bool paper = true;
    for (int k = 0; k < n_scenes; ++k) paper = paper && merf::paper_geometry(scenes[k]->desc);
    s->grid = paper ? (prec == MERF_PREC_FP16   ? resident_grid<1, merf::kGeoPaper>()
                       : prec == MERF_PREC_BF16 ? resident_grid<2, merf::kGeoPaper>()
                                                : resident_grid<0, merf::kGeoPaper>())
                    : (prec == MERF_PREC_FP16   ? resident_grid<1, merf::kGeoRuntime>()
                       : prec == MERF_PREC_BF16 ? resident_grid<2, merf::kGeoRuntime>()
                                                : resident_grid<0, merf::kGeoRuntime>());
    cudaError_t e = cudaMalloc(&s->d_pool, opts->pool_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_counter, 2 * sizeof(int));
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaMalloc(&s->d_work[b], sizeof(merf::ServeWork));
        if (e == cudaSuccess) e = cudaHostAlloc(&s->h_work[b], sizeof(merf::ServeWork), cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_iter[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_comp, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_copy, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        const bool oom = e == cudaErrorMemoryAllocation;
        cudaGetLastError();
        delete s;
        return merf::set_error(oom ? MERF_ERR_OOM : MERF_ERR_CUDA, "server resources: %s", cudaGetErrorString(e));
    }
    for (int b = 0; b < 2; ++b) {
        merf::ServeParams &P = s->params[b];
        memset(&P, 0, sizeof P);
        for (int k = 0; k < n_scenes; ++k) {
            merf::scene_views(scenes[k], P.scenes[k].fv, P.scenes[k].occ);
            P.scenes[k].mlp = (const float *)scenes[k]->mlp;
        }
        P.work = s->d_work[b];
        P.counter = s->d_counter + b;
        P.pool = s->d_pool;
        P.step = opts->step;
        P.t_term = opts->t_term;
        P.early_term = opts->early_term;
        memset(s->h_work[b], 0, sizeof(int) * 4);
        const merf_status st =
            paper ? (prec == MERF_PREC_FP16   ? capture<1, merf::kGeoPaper>(s, b)
                     : prec == MERF_PREC_BF16 ? capture<2, merf::kGeoPaper>(s, b)
                                              : capture<0, merf::kGeoPaper>(s, b))
                  : (prec == MERF_PREC_FP16   ? capture<1, merf::kGeoRuntime>(s, b)
                     : prec == MERF_PREC_BF16 ? capture<2, merf::kGeoRuntime>(s, b)
                                              : capture<0, merf::kGeoRuntime>(s, b));
        if (st != MERF_OK) {
            delete s;
            return st;
        }
    }
    merf_server *srv = new merf_server();
    srv->be = s;
    srv->sched = new merf::ServeScheduler(*s, n_scenes, opts->pool_bytes / sizeof(float), opts->max_tiles_per_iter,
                                          serve_err, opts->max_tiles_backlog);
    srv->sched->start();
    *out = srv;
    return merf::clear_error();
}

merf_status merf_server_submit(merf_server *srv, int scene, const merf_camera *cam, int W, int H, float *h_out,
                               uint64_t *req_id)
{
    if (!srv) return merf::set_error(MERF_ERR_INVALID_ARG, "srv is NULL");
    return srv->sched->submit(scene, cam, W, H, h_out, req_id);
}

merf_status merf_server_wait(merf_server *srv, uint64_t req_id, double timeout_s, double *latency_s)
{
    if (!srv) return merf::set_error(MERF_ERR_INVALID_ARG, "srv is NULL");
    return srv->sched->wait(req_id, timeout_s, latency_s);
}

merf_status merf_server_wait_timed(merf_server *srv, uint64_t req_id, double timeout_s, double *latency_s,
                                   merf_request_timing *timing)
{
    if (!srv) return merf::set_error(MERF_ERR_INVALID_ARG, "srv is NULL");
    return srv->sched->wait_timed(req_id, timeout_s, latency_s, timing);
}

merf_status merf_server_cancel(merf_server *srv, uint64_t req_id, int *cancelled)
{
    if (!srv) return merf::set_error(MERF_ERR_INVALID_ARG, "srv is NULL");
    return srv->sched->cancel(req_id, cancelled);
}

merf_status merf_server_get_stats(merf_server *srv, merf_server_stats *out)
{
    if (!srv) return merf::set_error(MERF_ERR_INVALID_ARG, "srv is NULL");
    return srv->sched->stats(out);
}

void merf_server_destroy(merf_server *srv)
{
    if (!srv) return;
    srv->sched->stop();
    delete srv->sched;          // releases the requests' events
    delete srv->be;
    delete srv;
}

}  // extern "C"
