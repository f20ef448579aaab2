// vi_server.cu -- a native inpainting server: requests queue in arrival
// order, are admitted while their device footprint (vi_footprint_bytes) fits
// the HBM budget and a worker slot is free, and each admitted request runs
// alone (vi_run) in a worker thread on a stream its context creates with a
// priority by size (smaller requests first), so the GPU interleaves them and a
// small request is not held to the pace of a large one. Device memory is
// stream-ordered in the library, so one request's allocation and release do
// not stall the others. Results are written to the caller's output buffer;
// every result is bit-identical to the same clip run alone.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "vi.h"
#include "vi_ctx.h"

namespace {

enum JobState { JOB_QUEUED = 0, JOB_RUNNING = 1, JOB_DONE = 2, JOB_FAILED = 3 };

struct Job {
    uint64_t ticket = 0;
    vi_config cfg{};
    const float *rgb = nullptr;
    const uint8_t *mask = nullptr;
    float *out = nullptr;
    int W = 0, H = 0, T = 0;
    int ptr_is_device = 0;
    size_t footprint = 0;
    int state = JOB_QUEUED;
    vi_status status = VI_OK;
    std::string err;
};

// priority by size: under 2M / 8M / 32M voxels the three highest, else 0
int size_priority(long long voxels)
{
    if (voxels < 2000000)
        return -3;
    if (voxels < 8000000)
        return -2;
    if (voxels < 32000000)
        return -1;
    return 0;
}

}  // namespace

struct vi_server {
    size_t budget = 0;
    int slots = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;        // queue, slots or memory changed; or stop
    std::condition_variable done_cv;   // a job finished
    std::deque<uint64_t> queue;
    std::map<uint64_t, Job> jobs;
    uint64_t next_ticket = 1;
    size_t used = 0;
    int running = 0;
    bool stop = false;
    std::vector<std::thread> workers;
};

namespace {

// Runs one admitted job (footprint fp) and, in one critical section, marks it
// finished and returns its memory and slot.
void run_job(vi_server *s, Job &job, size_t fp)
{
    cudaSetDevice(s->device);
    vi_config cfg = job.cfg;
    cfg.stream_priority = size_priority((long long)job.W * job.H * job.T);
    vi_ctx *ctx = nullptr;
    vi_status st = vi_ctx_create(&cfg, nullptr, &ctx);
    const char *err = nullptr;
    if (st == VI_OK)
        st = vi_upload(ctx, job.rgb, job.mask, job.W, job.H, job.T, job.ptr_is_device);
    if (st == VI_OK)
        st = vi_run(ctx);
    if (st == VI_OK)
        st = vi_fetch_result(ctx, job.out, job.ptr_is_device);
    // a device result is complete only once the context's stream has drained
    if (st == VI_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        st = VI_ERR_CUDA;
        err = cudaGetErrorString(cudaGetLastError());
    } else if (st != VI_OK) {
        err = ctx ? vi_last_error(ctx) : "vi_ctx_create failed";
    }
    std::string msg;
    try {
        msg = err ? err : "";   // copied before the context (which owns the text) goes
    } catch (...) {             // no room for the message: the status still says what failed
    }
    if (ctx)
        vi_ctx_destroy(ctx);
    std::lock_guard<std::mutex> lock(s->mu);
    job.status = st;
    job.err.swap(msg);
    job.state = st == VI_OK ? JOB_DONE : JOB_FAILED;
    s->used -= fp;
    --s->running;
    s->cv.notify_all();
    s->done_cv.notify_all();
}

void worker_loop(vi_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        // first come, first served: the head of the queue waits for memory
        s->cv.wait(lock, [s] {
            if (s->stop)
                return true;
            if (s->queue.empty())
                return false;
            const Job &j = s->jobs[s->queue.front()];
            return s->used + j.footprint <= s->budget;
        });
        if (s->stop && s->queue.empty())
            return;
        if (s->stop) {
            // fail the queued jobs on shutdown
            while (!s->queue.empty()) {
                Job &j = s->jobs[s->queue.front()];
                s->queue.pop_front();
                j.state = JOB_FAILED;
                j.status = VI_ERR_STATE;
                try {
                    j.err = "server destroyed";
                } catch (...) {
                }
            }
            s->done_cv.notify_all();
            return;
        }
        const uint64_t t = s->queue.front();
        s->queue.pop_front();
        Job &job = s->jobs[t];
        job.state = JOB_RUNNING;
        // once run_job marks the job finished, its owner may release it at
        // any time, so nothing of it is read afterwards
        const size_t fp = job.footprint;
        s->used += fp;
        ++s->running;
        lock.unlock();
        run_job(s, job, fp);
        lock.lock();
    }
}

}  // namespace

extern "C" {

vi_status vi_server_create(size_t hbm_budget, int max_slots, vi_server **out)
{
    if (!out || hbm_budget == 0 || max_slots <= 0 || max_slots > 256)
        return VI_ERR_ARG;
    *out = nullptr;
    int ndev = 0, dev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0 || cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return VI_ERR_NO_DEVICE;
    }
    vi_server *s = new (std::nothrow) vi_server();
    if (!s)
        return VI_ERR_OOM;
    s->budget = hbm_budget;
    s->slots = max_slots;
    s->device = dev;
    try {
        for (int i = 0; i < max_slots; ++i)
            s->workers.emplace_back(worker_loop, s);
    } catch (...) {
        vi_server_destroy(s);
        return VI_ERR_OOM;
    }
    *out = s;
    return VI_OK;
}

vi_status vi_server_submit(vi_server *s, const vi_config *cfg, const float *rgb, const uint8_t *mask, int W,
                           int H, int T, int ptr_is_device, float *rgb_out, uint64_t *ticket)
{
    if (!s || !rgb || !mask || !rgb_out || !ticket || W <= 0 || H <= 0 || T <= 0 ||
        (long long)W * H * T >= (1ll << 31))
        return VI_ERR_ARG;
    vi_config c;
    if (cfg)
        c = *cfg;
    else
        vi_config_default(&c);
    // the footprint bound does not depend on the hole size, so the mask is not scanned here
    const size_t fp = vi_footprint_bytes(&c, W, H, T, 0);
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop)
        return VI_ERR_STATE;
    if (fp > s->budget)
        return VI_ERR_TOO_LARGE;
    const uint64_t t = s->next_ticket;
    Job *jp = nullptr;
    try {
        jp = &s->jobs[t];
        s->queue.push_back(t);
    } catch (...) {
        s->jobs.erase(t);
        return VI_ERR_OOM;
    }
    ++s->next_ticket;
    Job &j = *jp;
    j.ticket = t;
    j.cfg = c;
    j.rgb = rgb;
    j.mask = mask;
    j.out = rgb_out;
    j.W = W;
    j.H = H;
    j.T = T;
    j.ptr_is_device = ptr_is_device;
    j.footprint = fp;
    *ticket = t;
    s->cv.notify_all();
    return VI_OK;
}

vi_status vi_server_poll(vi_server *s, uint64_t ticket, int *done)
{
    if (!s || !done)
        return VI_ERR_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end())
        return VI_ERR_ARG;
    const int st = it->second.state;
    *done = st == JOB_DONE ? 1 : (st == JOB_FAILED ? -1 : 0);
    return VI_OK;
}

vi_status vi_server_wait(vi_server *s, uint64_t ticket, double timeout_s, int *done)
{
    if (!s || !done)
        return VI_ERR_ARG;
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->jobs.find(ticket) == s->jobs.end())
        return VI_ERR_ARG;
    // looked up afresh on every wake-up: another thread may release the ticket meanwhile
    auto finished = [&] {
        auto f = s->jobs.find(ticket);
        return f == s->jobs.end() || f->second.state == JOB_DONE || f->second.state == JOB_FAILED;
    };
    if (timeout_s < 0)
        s->done_cv.wait(lock, finished);
    else
        s->done_cv.wait_for(lock, std::chrono::duration<double>(timeout_s), finished);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end())
        return VI_ERR_ARG;
    const int st = it->second.state;
    *done = st == JOB_DONE ? 1 : (st == JOB_FAILED ? -1 : 0);
    return VI_OK;
}

vi_status vi_server_release(vi_server *s, uint64_t ticket, char *err_buf, int err_cap)
{
    if (!s)
        return VI_ERR_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end())
        return VI_ERR_ARG;
    if (it->second.state != JOB_DONE && it->second.state != JOB_FAILED)
        return VI_ERR_STATE;
    const vi_status st = it->second.status;
    if (err_buf && err_cap > 0) {
        const std::string &e = it->second.err;
        const size_t n = std::min(e.size(), (size_t)err_cap - 1);
        e.copy(err_buf, n);
        err_buf[n] = '\0';
    }
    s->jobs.erase(it);
    return st;
}

vi_status vi_server_info(vi_server *s, int *queued, int *running, size_t *bytes_in_use)
{
    if (!s)
        return VI_ERR_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    if (queued)
        *queued = (int)s->queue.size();
    if (running)
        *running = s->running;
    if (bytes_in_use)
        *bytes_in_use = s->used;
    return VI_OK;
}

void vi_server_destroy(vi_server *s)
{
    if (!s)
        return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    for (std::thread &t : s->workers)
        if (t.joinable())
            t.join();
    delete s;
}

}  // extern "C"
