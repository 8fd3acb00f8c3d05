// Host stand-in for the serving form's device, for CPU tests of the scheduler
// (paper_2302_12249_b300/csrc/serve_sched.h -- the same code the CUDA server runs).
//
// An iteration runs its tiles on worker threads through a caller-supplied tile function that
// renders into a host "pool"; copying an image out is a memcpy.  A gate can hold iterations
// before their tiles run, so a test can act while requests are in flight, and a tile function
// that returns non-zero fails its iteration, standing in for a failed device launch.  Built by
// the tests with g++ and driven through this small C ABI.
#include <atomic>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "serve_sched.h"

// Render the pixels [x0, x0 + 16) x [y0, y0 + 8) (clipped to W x H) of one request into its
// image (H x W x 3 floats at its pool offset).  Non-zero: the tile failed.
typedef int (*host_tile_fn)(void *user, int scene, int W, int H, const float *cam, int x0, int y0, float *image);

namespace {

thread_local std::string g_err;

merf_status host_err(merf_status s, const char *msg)
{
    g_err = msg;
    return s;
}

class HostBackend final : public merf::ServeBackend {
public:
    HostBackend(size_t pool_floats, int workers, host_tile_fn fn, void *user)
        : pool_(pool_floats, 0.0f), workers_(workers < 1 ? 1 : workers), fn_(fn), user_(user)
    {
        for (int b = 0; b < 2; ++b) work_[b] = new merf::ServeWork();
    }

    ~HostBackend() override
    {
        drain();
        for (int b = 0; b < 2; ++b) delete work_[b];
    }

    merf::ServeWork *work(int b) override { return work_[b]; }

    bool launch(int b) override
    {
        join(b);
        state_[b].store(0);
        runner_[b] = std::thread([this, b] { run(b); });
        return true;
    }

    int poll_iter(int b) override
    {
        const int s = state_[b].load();
        if (s == 0) return 0;
        join(b);
        return s > 0 ? 1 : -1;
    }

    merf_status req_init(merf::ServeRequest &) override { return MERF_OK; }
    void req_free(merf::ServeRequest &) override {}

    bool copy_out(merf::ServeRequest &r) override
    {
        memcpy(r.h_out, pool_.data() + r.pool_off, r.floats * sizeof(float));
        return true;
    }

    int poll_copy(merf::ServeRequest &) override { return 1; }

    void drain() override
    {
        set_hold(false);
        join(0);
        join(1);
    }

    void set_hold(bool on)
    {
        {
            std::lock_guard<std::mutex> lk(mu_);
            hold_ = on;
        }
        cv_.notify_all();
    }

private:
    void join(int b)
    {
        if (runner_[b].joinable()) runner_[b].join();
    }

    void run(int b)
    {
        {
            std::unique_lock<std::mutex> lk(mu_);
            cv_.wait(lk, [this] { return !hold_; });
        }
        const merf::ServeWork &w = *work_[b];
        std::atomic<int> next{0};
        std::atomic<bool> bad{false};
        auto worker = [&] {
            for (;;) {
                const int t = next.fetch_add(1);
                if (t >= w.n_tiles) return;
                const uint32_t code = w.tiles[t];
                const merf::ServeReq &q = w.req[code >> 20];
                const int tl = (int)(code & 0xfffffu);
                const int x0 = (tl % q.tiles_x) * merf::kServeTileW, y0 = (tl / q.tiles_x) * merf::kServeTileH;
                if (fn_(user_, q.scene, q.W, q.H, q.cam, x0, y0, pool_.data() + q.out_off)) bad = true;
            }
        };
        std::vector<std::thread> ts;
        for (int k = 1; k < workers_; ++k) ts.emplace_back(worker);
        worker();
        for (auto &t : ts) t.join();
        state_[b].store(bad ? -1 : 1);
    }

    std::vector<float> pool_;
    const int workers_;
    host_tile_fn fn_;
    void *user_;
    merf::ServeWork *work_[2] = {nullptr, nullptr};
    std::thread runner_[2];
    std::atomic<int> state_[2] = {{0}, {0}};
    std::mutex mu_;
    std::condition_variable cv_;
    bool hold_ = false;
};

struct HostServer {
    HostBackend *be;
    merf::ServeScheduler *sched;
};

}  // namespace

extern "C" {

void *host_server_create(int n_scenes, size_t pool_bytes, int max_tiles_per_iter, int workers, host_tile_fn fn,
                         void *user, int max_tiles_backlog)
{
    HostServer *h = new HostServer();
    h->be = new HostBackend(pool_bytes / sizeof(float), workers, fn, user);
    h->sched = new merf::ServeScheduler(*h->be, n_scenes, pool_bytes / sizeof(float), max_tiles_per_iter, host_err,
                                        max_tiles_backlog);
    h->sched->start();
    return h;
}

int host_server_submit(void *p, int scene, const float *cam, int W, int H, float *out, uint64_t *id)
{
    return static_cast<HostServer *>(p)->sched->submit(scene, reinterpret_cast<const merf_camera *>(cam), W, H, out, id);
}

int host_server_wait(void *p, uint64_t id, double timeout_s, double *latency_s)
{
    return static_cast<HostServer *>(p)->sched->wait(id, timeout_s, latency_s);
}

int host_server_wait_timed(void *p, uint64_t id, double timeout_s, double *latency_s, merf_request_timing *t)
{
    return static_cast<HostServer *>(p)->sched->wait_timed(id, timeout_s, latency_s, t);
}

int host_server_cancel(void *p, uint64_t id, int *cancelled)
{
    return static_cast<HostServer *>(p)->sched->cancel(id, cancelled);
}

int host_server_stats(void *p, merf_server_stats *st) { return static_cast<HostServer *>(p)->sched->stats(st); }

void host_server_hold(void *p, int on) { static_cast<HostServer *>(p)->be->set_hold(on != 0); }

const char *host_server_last_error(void) { return g_err.c_str(); }

size_t host_stats_size(void) { return sizeof(merf_server_stats); }

void host_server_destroy(void *p)
{
    HostServer *h = static_cast<HostServer *>(p);
    h->be->set_hold(false);       // held iterations must run for the scheduler to finish
    h->sched->stop();
    delete h->sched;
    delete h->be;
    delete h;
}

}  // extern "C"
