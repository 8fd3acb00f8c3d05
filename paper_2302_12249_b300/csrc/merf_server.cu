// merf_server.cu -- the serving form: a continuous-batching render server (declared in merf.h).
//
// Host side: one server thread per server.  Requests wait in arrival order until their output
// image fits in the device output pool (a first-fit free list over one allocation); admitted
// requests are cut into 16 x 8 pixel tiles, and each iteration packs the oldest requests' next
// tiles -- any scene, any resolution -- into a work list of at most max_tiles_per_iter tiles.  An
// iteration is one launch of a captured CUDA graph (work-list upload, counter reset, persistent
// kernel).  Two work buffers and graphs alternate, so one iteration runs while the next is
// built; a request's last iteration completing starts the copy of its image to host memory on a
// second stream, and the copy's event completes the request.
//
// Device side: serve_kernel keeps one CTA per resident slot (SMs x CTAs per SM) and pulls tiles
// from the work list with an atomic counter, so long and short requests balance across SMs.  Each
// CTA renders its tile with the same march and deferred MLP as render_kernel; the MLP weights in
// shared memory are reloaded when a tile belongs to another scene.  There is no device-side wait.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "merf.h"
#include "render.cuh"
#include "scene.h"

namespace merf {

constexpr int kServeMaxScenes = 8;
constexpr int kServeMaxReq = 512;          // requests per iteration
constexpr int kServeMaxTiles = 1 << 16;    // tiles per iteration
constexpr int kServeMaxTilesPerReq = 1 << 20;

struct ServeReq {
    int32_t scene, W, H, tiles_x;
    unsigned long long out_off;            // float offset of the image in the pool
    int32_t pad[2];
    float cam[16];
};

struct ServeWork {
    int32_t n_tiles, n_req, pad0, pad1;
    ServeReq req[kServeMaxReq];
    uint32_t tiles[kServeMaxTiles];        // request index << 20 | tile index in the request
};

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
    const int n_tiles = P.work->n_tiles;
    int cur_scene = -1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(P.counter, 1);
        __syncthreads();
        const int tile = s_tile;
        if (tile >= n_tiles) break;
        const uint32_t code = P.work->tiles[tile];
        const ServeReq &R = P.work->req[code >> 20];
        const int sc = R.scene;
        if (sc != cur_scene) {          // uniform across the CTA
            ms.load(P.scenes[sc].mlp);
            __syncthreads();
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
        deferred_mlp<kPrec>(ms, r, inside, h);
        if (inside) {
            float *o = P.pool + R.out_off + ((size_t)j * R.W + i) * 3;
            o[0] = r.cd[0] + h[0];
            o[1] = r.cd[1] + h[1];
            o[2] = r.cd[2] + h[2];
        }
        __syncthreads();                // s_tile and the weights are reused next iteration
    }
}

}  // namespace merf

namespace {

using Clock = std::chrono::steady_clock;

double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

// First-fit free list over [0, capacity) (units: floats, 64-float = 256-byte granules).
class Pool {
public:
    explicit Pool(size_t cap = 0) : cap_(cap) { if (cap) free_[0] = cap; }
    bool alloc(size_t n, size_t &off)
    {
        n = round(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            off = it->first;
            const size_t rest = it->second - n;
            free_.erase(it);
            if (rest) free_[off + n] = rest;
            used_ += n;
            peak_ = std::max(peak_, used_);
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        n = round(n);
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t capacity() const { return cap_; }
    size_t peak() const { return peak_; }
    static size_t round(size_t n) { return (n + 63) & ~(size_t)63; }

private:
    std::map<size_t, size_t> free_;
    size_t cap_ = 0, used_ = 0, peak_ = 0;
};

enum ReqState { kPending, kActive, kScheduled, kCopying, kDone, kFailed };

struct Req {
    uint64_t id;
    int scene, W, H, tiles_x, tiles_total, tiles_next = 0;
    float cam[16];
    float *h_out;
    size_t floats, pool_off = 0;
    double t_submit = 0, t_done = 0;
    ReqState state = kPending;
    cudaEvent_t copy_ev = nullptr;
    merf_status status = MERF_OK;
};

}  // namespace

struct merf_server {
    merf_server_opts opts;
    int device = 0, n_scenes = 0, grid = 0;
    merf::ServeParams params[2];
    float *d_pool = nullptr;
    merf::ServeWork *h_work[2] = {nullptr, nullptr}, *d_work[2] = {nullptr, nullptr};
    int *d_counter = nullptr;
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaStream_t s_comp = nullptr, s_copy = nullptr;
    cudaEvent_t ev_iter[2] = {nullptr, nullptr};
    bool busy[2] = {false, false};
    std::vector<Req *> finishing[2];
    Pool pool;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> pending, active;
    std::vector<Req *> copying;
    std::unordered_map<uint64_t, Req *> reqs;
    uint64_t next_id = 1;
    bool stopping = false;
    merf_status fatal = MERF_OK;
    std::thread th;
    merf_server_stats st{};
    int admitted = 0;

    void fail_all(merf_status s)
    {
        fatal = s;
        for (auto &kv : reqs)
            if (kv.second->state != kDone) {
                kv.second->state = kFailed;
                kv.second->status = s;
            }
        cv_done.notify_all();
    }

    // Pack the oldest admitted requests' next tiles into work buffer b (mutex held).
    void build(int b)
    {
        merf::ServeWork &w = *h_work[b];
        int nt = 0, nr = 0;
        const int budget = opts.max_tiles_per_iter;
        while (!active.empty() && nt < budget && nr < merf::kServeMaxReq) {
            Req *r = active.front();
            merf::ServeReq &q = w.req[nr];
            q.scene = r->scene;
            q.W = r->W;
            q.H = r->H;
            q.tiles_x = r->tiles_x;
            q.out_off = r->pool_off;
            memcpy(q.cam, r->cam, sizeof q.cam);
            const int take = std::min(budget - nt, r->tiles_total - r->tiles_next);
            for (int t = 0; t < take; ++t) w.tiles[nt + t] = ((uint32_t)nr << 20) | (uint32_t)(r->tiles_next + t);
            nt += take;
            r->tiles_next += take;
            ++nr;
            if (r->tiles_next == r->tiles_total) {
                r->state = kScheduled;
                finishing[b].push_back(r);
                active.pop_front();
            }
        }
        w.n_tiles = nt;
        w.n_req = nr;
        st.tiles += nt;
    }

    void loop()
    {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            bool progress = false;
            // iterations that finished: start the copies of the requests they completed
            for (int b = 0; b < 2; ++b) {
                if (!busy[b]) continue;
                const cudaError_t q = cudaEventQuery(ev_iter[b]);
                if (q == cudaErrorNotReady) continue;
                if (q != cudaSuccess) { fail_all(MERF_ERR_CUDA); return; }
                busy[b] = false;
                for (Req *r : finishing[b]) {
                    const cudaError_t e = cudaMemcpyAsync(r->h_out, d_pool + r->pool_off, r->floats * sizeof(float),
                                                          cudaMemcpyDeviceToHost, s_copy);
                    if (e != cudaSuccess || cudaEventRecord(r->copy_ev, s_copy) != cudaSuccess) {
                        fail_all(MERF_ERR_CUDA);
                        return;
                    }
                    r->state = kCopying;
                    copying.push_back(r);
                }
                finishing[b].clear();
                progress = true;
            }
            // copies that landed: the request is complete
            for (size_t k = 0; k < copying.size();) {
                Req *r = copying[k];
                const cudaError_t q = cudaEventQuery(r->copy_ev);
                if (q == cudaErrorNotReady) { ++k; continue; }
                if (q != cudaSuccess) { fail_all(MERF_ERR_CUDA); return; }
                r->t_done = now_s();
                r->state = kDone;
                pool.release(r->pool_off, r->floats);
                --admitted;
                st.completed += 1;
                st.rays += (unsigned long long)r->W * r->H;
                copying[k] = copying.back();
                copying.pop_back();
                cv_done.notify_all();
                progress = true;
            }
            // admission by free pool memory, in arrival order
            while (!pending.empty()) {
                Req *r = pending.front();
                if (!pool.alloc(r->floats, r->pool_off)) break;
                r->state = kActive;
                active.push_back(r);
                pending.pop_front();
                ++admitted;
                st.peak_admitted = std::max(st.peak_admitted, admitted);
                progress = true;
            }
            // launch iterations into free buffers
            for (int b = 0; b < 2 && !active.empty(); ++b) {
                if (busy[b]) continue;
                build(b);
                if (cudaGraphLaunch(exec[b], s_comp) != cudaSuccess || cudaEventRecord(ev_iter[b], s_comp) != cudaSuccess) {
                    fail_all(MERF_ERR_CUDA);
                    return;
                }
                busy[b] = true;
                st.iterations += 1;
                progress = true;
            }
            if (stopping && pending.empty() && active.empty() && copying.empty() && !busy[0] && !busy[1]) return;
            if (!progress) cv_work.wait_for(lk, std::chrono::microseconds(50));
        }
    }
};

namespace merf {
unsigned int take_server_status()
{
#ifdef MERF_DEBUG_BOUNDS
    unsigned int word = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&word, g_status, sizeof word) != cudaSuccess) return 0;
    cudaMemcpyToSymbol(g_status, &zero, sizeof zero);
    return word;
#else
    return 0;
#endif
}
}  // namespace merf

namespace {

template <int kPrec, int kGeo>
merf_status capture(merf_server *s, int b)
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

template <int kPrec, int kGeo>
int resident_grid()
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, merf::serve_kernel<kPrec, kGeo>, merf::kThreads, 0);
    return std::max(1, sms) * std::max(1, per);
}

void release(merf_server *s)
{
    for (int b = 0; b < 2; ++b) {
        if (s->exec[b]) cudaGraphExecDestroy(s->exec[b]);
        if (s->graph[b]) cudaGraphDestroy(s->graph[b]);
        if (s->ev_iter[b]) cudaEventDestroy(s->ev_iter[b]);
        if (s->h_work[b]) cudaFreeHost(s->h_work[b]);
        if (s->d_work[b]) cudaFree(s->d_work[b]);
    }
    if (s->d_counter) cudaFree(s->d_counter);
    if (s->d_pool) cudaFree(s->d_pool);
    if (s->s_comp) cudaStreamDestroy(s->s_comp);
    if (s->s_copy) cudaStreamDestroy(s->s_copy);
    for (auto &kv : s->reqs) {
        if (kv.second->copy_ev) cudaEventDestroy(kv.second->copy_ev);
        delete kv.second;
    }
    delete s;
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
    if (opts->reserved != 0) return merf::set_error(MERF_ERR_INVALID_ARG, "reserved must be 0");
    if (opts->max_tiles_per_iter < 1 || opts->max_tiles_per_iter > merf::kServeMaxTiles)
        return merf::set_error(MERF_ERR_INVALID_ARG, "max_tiles_per_iter %d not in [1, %d]", opts->max_tiles_per_iter,
                               merf::kServeMaxTiles);
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
    merf_server *s = new merf_server();
    s->opts = *opts;
    s->n_scenes = n_scenes;
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
        release(s);
        return merf::set_error(oom ? MERF_ERR_OOM : MERF_ERR_CUDA, "server resources: %s", cudaGetErrorString(e));
    }
    s->pool = Pool(opts->pool_bytes / sizeof(float) & ~(size_t)63);
    s->st.pool_bytes = s->pool.capacity() * sizeof(float);
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
            release(s);
            return st;
        }
    }
    s->th = std::thread([s] { s->loop(); });
    *out = s;
    return merf::clear_error();
}

merf_status merf_server_submit(merf_server *srv, int scene, const merf_camera *cam, int W, int H, float *h_out,
                               uint64_t *req_id)
{
    if (!srv || !cam || !h_out || !req_id) return merf::set_error(MERF_ERR_INVALID_ARG, "NULL argument");
    if (scene < 0 || scene >= srv->n_scenes) return merf::set_error(MERF_ERR_INVALID_ARG, "scene %d out of range", scene);
    if (W < 1 || H < 1 || W > 16384 || H > 16384) return merf::set_error(MERF_ERR_INVALID_ARG, "W %d / H %d invalid", W, H);
    const int tx = (W + merf::kTileW - 1) / merf::kTileW, ty = (H + merf::kTileH - 1) / merf::kTileH;
    if ((long long)tx * ty > merf::kServeMaxTilesPerReq)
        return merf::set_error(MERF_ERR_INVALID_ARG, "request of %d x %d tiles is too large", tx, ty);
    for (int t = 0; t < 12; ++t)
        if (!(cam->c2w[t] == cam->c2w[t]) || cam->c2w[t] > 1e30f || cam->c2w[t] < -1e30f)
            return merf::set_error(MERF_ERR_INVALID_ARG, "camera not finite");
    if (!(cam->fx != 0.0f) || !(cam->fy != 0.0f)) return merf::set_error(MERF_ERR_INVALID_ARG, "camera intrinsics");
    const size_t floats = (size_t)W * H * 3;
    if (Pool::round(floats) > srv->pool.capacity())
        return merf::set_error(MERF_ERR_OOM, "a %d x %d image needs %zu bytes, the pool holds %zu", W, H,
                               floats * sizeof(float), srv->pool.capacity() * sizeof(float));
    Req *r = new Req();
    r->scene = scene;
    r->W = W;
    r->H = H;
    r->tiles_x = tx;
    r->tiles_total = tx * ty;
    memcpy(r->cam, cam, sizeof r->cam);
    r->h_out = h_out;
    r->floats = floats;
    if (cudaEventCreateWithFlags(&r->copy_ev, cudaEventDisableTiming) != cudaSuccess) {
        delete r;
        return merf::set_error(MERF_ERR_CUDA, "event creation failed");
    }
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->fatal != MERF_OK || srv->stopping) {
            cudaEventDestroy(r->copy_ev);
            delete r;
            return merf::set_error(srv->fatal != MERF_OK ? srv->fatal : MERF_ERR_INVALID_ARG, "server not accepting work");
        }
        r->id = srv->next_id++;
        r->t_submit = now_s();
        srv->pending.push_back(r);
        srv->reqs[r->id] = r;
        srv->st.submitted += 1;
        *req_id = r->id;
    }
    srv->cv_work.notify_one();
    return merf::clear_error();
}

merf_status merf_server_wait(merf_server *srv, uint64_t req_id, double timeout_s, double *latency_s)
{
    if (!srv) return merf::set_error(MERF_ERR_INVALID_ARG, "srv is NULL");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(req_id);
    if (it == srv->reqs.end()) return merf::set_error(MERF_ERR_INVALID_ARG, "unknown request %llu", (unsigned long long)req_id);
    Req *r = it->second;
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(std::max(0.0, timeout_s)));
    if (!srv->cv_done.wait_until(lk, deadline, [r] { return r->state == kDone || r->state == kFailed; }))
        return merf::set_error(MERF_ERR_TIMEOUT, "request %llu not complete after %.3f s", (unsigned long long)req_id,
                               timeout_s);
    const merf_status st = r->state == kDone ? MERF_OK : r->status;
    if (latency_s) *latency_s = r->t_done - r->t_submit;
    srv->reqs.erase(it);
    cudaEventDestroy(r->copy_ev);
    delete r;
    if (st != MERF_OK) return merf::set_error(st, "request failed on the device");
    return merf::clear_error();
}

merf_status merf_server_get_stats(merf_server *srv, merf_server_stats *out)
{
    if (!srv || !out) return merf::set_error(MERF_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->st;
    out->peak_pool_bytes = srv->pool.peak() * sizeof(float);
    return merf::clear_error();
}

void merf_server_destroy(merf_server *srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stopping = true;
    }
    srv->cv_work.notify_all();
    if (srv->th.joinable()) srv->th.join();
    cudaStreamSynchronize(srv->s_comp);
    cudaStreamSynchronize(srv->s_copy);
    release(srv);
}

}  // extern "C"
