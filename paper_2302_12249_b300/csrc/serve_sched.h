// serve_sched.h -- the scheduler of the serving form (merf_server_*, declared in merf.h):
// admission by output-pool memory, continuous batching of pixel tiles into iterations,
// completion and cancellation.
//
// Plain C++ with no CUDA.  The scheduler reaches the device only through ServeBackend: run the
// iteration built in slot b, poll it, copy a finished image out, poll the copy.  merf_server.cu
// implements the backend with captured CUDA graphs, events and a copy stream; a host stand-in
// whose iterations run tiles on threads drives the same scheduler on a machine without a GPU.
//
// Requests wait in arrival order until their image fits in the free part of the output pool (a
// first-fit free list over 256-byte granules).  Admitted requests are cut into 16 x 8 pixel
// tiles, and each iteration packs the oldest requests' next tiles -- any scene, any resolution --
// into a work list of at most max_tiles_per_iter tiles.  Two iteration slots alternate, so one
// iteration runs while the next is built.  Every request counts the iterations in flight that
// carry its tiles: when the last of them completes and all its tiles have run, its image is
// copied to its host buffer, and it completes when the copy lands.  Cancellation withdraws a
// request that is not yet being copied out; its pool space returns to the free list only once no
// iteration in flight can still write it, and its host buffer is never written.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "merf.h"

namespace merf {

constexpr int kServeTileW = 16, kServeTileH = 8;   // pixels of one tile (one CTA of 128 rays)
constexpr int kServeMaxScenes = 8;
constexpr int kServeMaxReq = 512;                  // requests per iteration
constexpr int kServeMaxTiles = 1 << 16;            // tiles per iteration
constexpr int kServeMaxTilesPerReq = 1 << 20;

// One request's entry in an iteration's work list (read by the device).
struct ServeReq {
    int32_t scene, W, H, tiles_x;
    unsigned long long out_off;            // float offset of the image in the pool
    int32_t pad[2];
    float cam[16];
};

// An iteration's work list: tiles[t] = request index << 20 | tile index within the request.
struct ServeWork {
    int32_t n_tiles, n_req, pad0, pad1;
    ServeReq req[kServeMaxReq];
    uint32_t tiles[kServeMaxTiles];
};

// First-fit free list over [0, capacity) (units: floats, 64-float = 256-byte granules).
class ServePool {
public:
    explicit ServePool(size_t cap = 0) : cap_(cap) { if (cap) free_[0] = cap; }
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
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }
    static size_t round(size_t n) { return (n + 63) & ~(size_t)63; }

private:
    std::map<size_t, size_t> free_;
    size_t cap_ = 0, used_ = 0, peak_ = 0;
};

enum ServeState { kPending, kActive, kScheduled, kCancelling, kCopying, kDone, kFailed };

struct ServeRequest {
    uint64_t id = 0;
    int scene = 0, W = 0, H = 0, tiles_x = 0, tiles_total = 0, tiles_next = 0;
    int inflight = 0;                      // iterations in flight that carry tiles of this request
    float cam[16];
    float *h_out = nullptr;
    size_t floats = 0, pool_off = 0;
    double t_submit = 0, t_done = 0;
    double t_admit = 0, t_launch = 0, t_rendered = 0;   // pool admission, first tiles launched, last tiles done
    ServeState state = kPending;
    merf_status status = MERF_OK;
    void *dev = nullptr;                   // the backend's per-request handle
};

// What the scheduler needs from the device.  Poll results: 1 complete, 0 still running, -1 failed.
class ServeBackend {
public:
    virtual ~ServeBackend() = default;
    virtual void thread_init() {}                               // on the server thread, first
    virtual ServeWork *work(int b) = 0;                         // host work list of slot b
    virtual bool launch(int b) = 0;                             // run the iteration built in slot b
    virtual int poll_iter(int b) = 0;
    virtual merf_status req_init(ServeRequest &r) = 0;          // per-request resources
    virtual void req_free(ServeRequest &r) = 0;
    virtual bool copy_out(ServeRequest &r) = 0;                 // pool image -> r.h_out
    virtual int poll_copy(ServeRequest &r) = 0;
    virtual void drain() {}                                     // wait for all device work
};

// Receives every call's outcome: (status, message), message "" on success.
using ServeErrFn = merf_status (*)(merf_status, const char *);

class ServeScheduler {
public:
    using Clock = std::chrono::steady_clock;

    ServeScheduler(ServeBackend &be, int n_scenes, size_t pool_floats, int max_tiles_per_iter, ServeErrFn err,
                   int max_tiles_backlog = 0)
        : be_(be), err_(err), n_scenes_(n_scenes), max_tiles_(max_tiles_per_iter),
          max_tiles_backlog_(max_tiles_backlog > max_tiles_per_iter ? max_tiles_backlog : max_tiles_per_iter),
          pool_(pool_floats & ~(size_t)63)
    {
        st_.pool_bytes = pool_.capacity() * sizeof(float);
    }

    ~ServeScheduler()
    {
        stop();
        for (auto &kv : reqs_) {
            be_.req_free(*kv.second);
            delete kv.second;
        }
    }

    void start() { th_ = std::thread([this] { loop(); }); }

    // Finish every submitted request and join the server thread.
    void stop()
    {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stopping_ = true;
        }
        cv_work_.notify_all();
        if (th_.joinable()) th_.join();
        be_.drain();
    }

    merf_status submit(int scene, const merf_camera *cam, int W, int H, float *h_out, uint64_t *req_id)
    {
        if (!cam || !h_out || !req_id) return fail(MERF_ERR_INVALID_ARG, "NULL argument");
        if (scene < 0 || scene >= n_scenes_) return fail(MERF_ERR_INVALID_ARG, "scene %d out of range", scene);
        if (W < 1 || H < 1 || W > 16384 || H > 16384) return fail(MERF_ERR_INVALID_ARG, "W %d / H %d invalid", W, H);
        const int tx = (W + kServeTileW - 1) / kServeTileW, ty = (H + kServeTileH - 1) / kServeTileH;
        if ((long long)tx * ty > kServeMaxTilesPerReq)
            return fail(MERF_ERR_INVALID_ARG, "request of %d x %d tiles is too large", tx, ty);
        for (int t = 0; t < 12; ++t)
            if (!(cam->c2w[t] == cam->c2w[t]) || cam->c2w[t] > 1e30f || cam->c2w[t] < -1e30f)
                return fail(MERF_ERR_INVALID_ARG, "camera not finite");
        if (!(cam->fx != 0.0f) || !(cam->fy != 0.0f)) return fail(MERF_ERR_INVALID_ARG, "camera intrinsics");
        const size_t floats = (size_t)W * H * 3;
        if (ServePool::round(floats) > pool_.capacity())
            return fail(MERF_ERR_OOM, "a %d x %d image needs %zu bytes, the pool holds %zu", W, H,
                        floats * sizeof(float), pool_.capacity() * sizeof(float));
        ServeRequest *r = new ServeRequest();
        r->scene = scene;
        r->W = W;
        r->H = H;
        r->tiles_x = tx;
        r->tiles_total = tx * ty;
        memcpy(r->cam, cam, sizeof r->cam);
        r->h_out = h_out;
        r->floats = floats;
        const merf_status rs = be_.req_init(*r);
        if (rs != MERF_OK) {
            delete r;
            return fail(rs, "request resources could not be created");
        }
        {
            std::lock_guard<std::mutex> lk(mu_);
            if (fatal_ != MERF_OK || stopping_) {
                be_.req_free(*r);
                delete r;
                return fail(fatal_ != MERF_OK ? fatal_ : MERF_ERR_INVALID_ARG, "server not accepting work");
            }
            r->id = next_id_++;
            r->t_submit = now_s();
            pending_.push_back(r);
            reqs_[r->id] = r;
            st_.submitted += 1;
            *req_id = r->id;
        }
        cv_work_.notify_one();
        return err_(MERF_OK, "");
    }

    merf_status wait(uint64_t req_id, double timeout_s, double *latency_s)
    {
        return wait_timed(req_id, timeout_s, latency_s, nullptr);
    }

    // wait, and on completion the request's phases (merf_request_timing; may be NULL)
    merf_status wait_timed(uint64_t req_id, double timeout_s, double *latency_s, merf_request_timing *timing)
    {
        std::unique_lock<std::mutex> lk(mu_);
        auto it = reqs_.find(req_id);
        if (it == reqs_.end()) return fail(MERF_ERR_INVALID_ARG, "unknown request %llu", (unsigned long long)req_id);
        ServeRequest *r = it->second;
        const auto deadline =
            Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(std::max(0.0, timeout_s)));
        if (!cv_done_.wait_until(lk, deadline, [r] { return r->state == kDone || r->state == kFailed; }))
            return fail(MERF_ERR_TIMEOUT, "request %llu not complete after %.3f s", (unsigned long long)req_id, timeout_s);
        const merf_status st = r->state == kDone ? MERF_OK : r->status;
        if (latency_s) *latency_s = r->t_done - r->t_submit;
        if (timing) {
            // phases end where the next begins; a request cancelled early has no later phases
            const double a = r->t_admit > 0 ? r->t_admit : r->t_done, l = r->t_launch > 0 ? r->t_launch : a,
                         e = r->t_rendered > 0 ? r->t_rendered : l;
            timing->total_s = r->t_done - r->t_submit;
            timing->admit_s = a - r->t_submit;
            timing->queue_s = l - a;
            timing->render_s = e - l;
            timing->copy_s = r->t_done - e;
        }
        reqs_.erase(it);
        be_.req_free(*r);
        delete r;
        if (st == MERF_ERR_CANCELLED) return fail(st, "request %llu was cancelled", (unsigned long long)req_id);
        if (st != MERF_OK) return fail(st, "request %llu failed on the device", (unsigned long long)req_id);
        return err_(MERF_OK, "");
    }

    // Withdraw a request that is not yet being copied out (*cancelled = 1); one whose image is
    // already on its way to host memory, or complete, is left to finish (*cancelled = 0).
    merf_status cancel(uint64_t req_id, int *cancelled)
    {
        if (!cancelled) return fail(MERF_ERR_INVALID_ARG, "NULL argument");
        *cancelled = 0;
        {
            std::lock_guard<std::mutex> lk(mu_);
            auto it = reqs_.find(req_id);
            if (it == reqs_.end()) return fail(MERF_ERR_INVALID_ARG, "unknown request %llu", (unsigned long long)req_id);
            ServeRequest *r = it->second;
            switch (r->state) {
            case kPending:                               // never admitted: nothing reserved
                pending_.erase(std::find(pending_.begin(), pending_.end(), r));
                retire_cancelled(r, false);
                *cancelled = 1;
                break;
            case kActive:                                // admitted, tiles still to schedule
                active_.erase(std::find(active_.begin(), active_.end(), r));
                if (r->inflight == 0) retire_cancelled(r, true);
                else r->state = kCancelling;
                *cancelled = 1;
                break;
            case kScheduled:                             // every tile issued, iterations running
                r->state = kCancelling;
                *cancelled = 1;
                break;
            default:                                     // being copied out, done or failed
                break;
            }
            if (*cancelled) st_.cancelled += 1;
        }
        cv_work_.notify_one();
        return err_(MERF_OK, "");
    }

    merf_status stats(merf_server_stats *out)
    {
        if (!out) return fail(MERF_ERR_INVALID_ARG, "NULL argument");
        std::lock_guard<std::mutex> lk(mu_);
        *out = st_;
        out->peak_pool_bytes = pool_.peak() * sizeof(float);
        out->pool_used_bytes = pool_.used() * sizeof(float);
        out->admitted = admitted_;
        out->queued = (int32_t)pending_.size();
        return err_(MERF_OK, "");
    }

private:
    static double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

    merf_status fail(merf_status s, const char *fmt, ...)
    {
        char buf[256];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        return err_(s, buf);
    }

    // (mutex held) the request ends as cancelled; its pool space, if it holds some, is free again
    void retire_cancelled(ServeRequest *r, bool holds_pool)
    {
        if (holds_pool) {
            pool_.release(r->pool_off, r->floats);
            --admitted_;
        }
        r->state = kFailed;
        r->status = MERF_ERR_CANCELLED;
        r->t_done = now_s();
        cv_done_.notify_all();
    }

    void fail_all(merf_status s)
    {
        fatal_ = s;
        for (auto &kv : reqs_)
            if (kv.second->state != kDone && kv.second->state != kFailed) {
                kv.second->state = kFailed;
                kv.second->status = s;
                kv.second->t_done = now_s();
            }
        cv_done_.notify_all();
    }

    // (mutex held) tiles the next iteration may carry: max_tiles_, or, while the admitted and queued
    // requests hold more than twice that many tiles not yet scheduled, up to max_tiles_backlog_
    // (half the backlog at most): under load, fewer and larger iterations spend less on each
    // iteration's launch and uneven finish, and latency is queueing then anyway
    int iteration_cap() const
    {
        if (max_tiles_backlog_ <= max_tiles_) return max_tiles_;
        long long backlog = 0;
        for (const ServeRequest *r : active_) backlog += r->tiles_total - r->tiles_next;
        for (const ServeRequest *r : pending_) backlog += r->tiles_total;
        if (backlog <= 2LL * max_tiles_) return max_tiles_;
        return (int)std::min<long long>(max_tiles_backlog_, std::max<long long>(max_tiles_, backlog / 2));
    }

    // (mutex held) pack the oldest admitted requests' next tiles into slot b's work list
    void build(int b)
    {
        ServeWork &w = *be_.work(b);
        int nt = 0, nr = 0;
        const int cap = iteration_cap();
        while (!active_.empty() && nt < cap && nr < kServeMaxReq) {
            ServeRequest *r = active_.front();
            ServeReq &q = w.req[nr];
            q.scene = r->scene;
            q.W = r->W;
            q.H = r->H;
            q.tiles_x = r->tiles_x;
            q.out_off = r->pool_off;
            memcpy(q.cam, r->cam, sizeof q.cam);
            const int take = std::min(cap - nt, r->tiles_total - r->tiles_next);
            if (r->tiles_next == 0) r->t_launch = now_s();          // its first tiles: this iteration
            for (int t = 0; t < take; ++t) w.tiles[nt + t] = ((uint32_t)nr << 20) | (uint32_t)(r->tiles_next + t);
            nt += take;
            r->tiles_next += take;
            r->inflight += 1;
            carried_[b].push_back(r);
            ++nr;
            if (r->tiles_next == r->tiles_total) {
                r->state = kScheduled;
                active_.pop_front();
            }
        }
        w.n_tiles = nt;
        w.n_req = nr;
        st_.tiles += nt;
    }

    void loop()
    {
        be_.thread_init();
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            bool progress = false;
            // iterations that finished: requests none of whose tiles are still running
            for (int b = 0; b < 2; ++b) {
                if (!busy_[b]) continue;
                const int q = be_.poll_iter(b);
                if (q == 0) continue;
                if (q < 0) { fail_all(MERF_ERR_CUDA); return; }
                busy_[b] = false;
                for (ServeRequest *r : carried_[b]) {
                    if (--r->inflight > 0) continue;
                    if (r->state == kCancelling) {
                        retire_cancelled(r, true);
                    } else if (r->state == kScheduled) {
                        r->t_rendered = now_s();
                        if (!be_.copy_out(*r)) { fail_all(MERF_ERR_CUDA); return; }
                        r->state = kCopying;
                        copying_.push_back(r);
                    }
                }
                carried_[b].clear();
                progress = true;
            }
            // copies that landed: the request is complete
            for (size_t k = 0; k < copying_.size();) {
                ServeRequest *r = copying_[k];
                const int q = be_.poll_copy(*r);
                if (q == 0) { ++k; continue; }
                if (q < 0) { fail_all(MERF_ERR_CUDA); return; }
                r->t_done = now_s();
                r->state = kDone;
                pool_.release(r->pool_off, r->floats);
                --admitted_;
                st_.completed += 1;
                st_.rays += (unsigned long long)r->W * r->H;
                copying_[k] = copying_.back();
                copying_.pop_back();
                cv_done_.notify_all();
                progress = true;
            }
            // admission by free pool memory, in arrival order
            while (!pending_.empty()) {
                ServeRequest *r = pending_.front();
                if (!pool_.alloc(r->floats, r->pool_off)) break;
                r->state = kActive;
                r->t_admit = now_s();
                active_.push_back(r);
                pending_.pop_front();
                ++admitted_;
                st_.peak_admitted = std::max(st_.peak_admitted, admitted_);
                progress = true;
            }
            // launch iterations into free slots
            for (int b = 0; b < 2 && !active_.empty(); ++b) {
                if (busy_[b]) continue;
                build(b);
                if (!be_.launch(b)) { fail_all(MERF_ERR_CUDA); return; }
                busy_[b] = true;
                st_.iterations += 1;
                progress = true;
            }
            if (stopping_ && pending_.empty() && active_.empty() && copying_.empty() && !busy_[0] && !busy_[1]) return;
            if (!progress) cv_work_.wait_for(lk, std::chrono::microseconds(50));
        }
    }

    ServeBackend &be_;
    ServeErrFn err_;
    const int n_scenes_, max_tiles_, max_tiles_backlog_;
    ServePool pool_;

    std::mutex mu_;
    std::condition_variable cv_work_, cv_done_;
    std::deque<ServeRequest *> pending_, active_;
    std::vector<ServeRequest *> copying_, carried_[2];
    std::unordered_map<uint64_t, ServeRequest *> reqs_;
    bool busy_[2] = {false, false};
    uint64_t next_id_ = 1;
    bool stopping_ = false;
    merf_status fatal_ = MERF_OK;
    std::thread th_;
    merf_server_stats st_{};
    int admitted_ = 0;
};

}  // namespace merf
