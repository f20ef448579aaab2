// vi_batch.cu -- many clips, one launch per step.
//
// A batch holds several clips (each a vi_ctx on the batch's stream, with its
// own pyramid, levels, seed and stopping rule). Clips are prepared when they
// are added (pyramid, shift-map initialisation, onion peel); then every call
// to vi_batch_step runs one search/reconstruction iteration (Algorithm 4's
// inner loop) for every clip that is still iterating, whatever its level:
// one rescore launch, n_pm PatchMatch launches and one vote launch cover the
// targets and occluded voxels of all those clips together (a descriptor per
// clip, prefix sums of their target and voxel counts, persistent grids).
// After the round the host reads each clip's change e and moves each clip on:
// next iteration, level transition, or final step. Clips may be added and
// removed between rounds (continuous batching).
//
// A clip's result is bit-identical to running it alone with vi_run: the batch
// kernels evaluate each target and voxel exactly as the single-clip ones do,
// and e is reduced per clip with the same fixed-order sum.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "vi_ctx.h"

using namespace vi;

namespace {

enum ClipState { CLIP_ITERATING = 1, CLIP_DONE = 2, CLIP_FAILED = 3 };

struct Entry {
    vi_ctx *ctx = nullptr;
    int id = 0;
    int state = CLIP_ITERATING;
    int level = 0;
    int outer = 0;
    float e = INFINITY;
    vi_status err = VI_OK;
};

}  // namespace

struct vi_batch {
    vi_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    std::vector<Entry> clips;
    int next_id = 0;

    int cap = 0;                       // clips the descriptor buffers hold
    BatchClip *d_clips = nullptr, *h_clips = nullptr;
    // targets (cap + 1), holes (cap + 1), chunks of the change sums (cap + 1)
    int *d_prefix = nullptr, *h_prefix = nullptr;
    double *d_e = nullptr, *h_e = nullptr;
    float *d_change = nullptr;
    long long change_cap = 0;
    double *d_chunks = nullptr;
    int chunks_cap = 0;
    // rescore evals, step evals, FP32 voxels gathered, FP16 voxels gathered,
    // screened, passed
    unsigned long long *counters = nullptr;
    unsigned long long rounds = 0;
    unsigned long long removed_evals = 0;            // own evaluations of removed clips

    bool profiling = false;                          // events around the step launches
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
    size_t events_used = 0;
    double step_ms = 0.0;
};

namespace {

vi_status bfail(vi_batch *b, vi_status st, const std::string &msg)
{
    if (b)
        b->err = msg;
    return st;
}

#define BCK(call)                                                                                 \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return bfail(b, VI_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
    } while (0)

Entry *find(vi_batch *b, int id)
{
    for (Entry &e : b->clips)
        if (e.id == id)
            return &e;
    return nullptr;
}

vi_status ensure_capacity(vi_batch *b, int n, long long holes, int chunks = 0)
{
    if (n > b->cap) {
        int cap = std::max(n, std::max(16, 2 * b->cap));
        if (b->d_clips) cudaFreeAsync(b->d_clips, b->stream);
        if (b->h_clips) cudaFreeHost(b->h_clips);
        if (b->d_prefix) cudaFreeAsync(b->d_prefix, b->stream);
        if (b->h_prefix) cudaFreeHost(b->h_prefix);
        if (b->d_e) cudaFreeAsync(b->d_e, b->stream);
        if (b->h_e) cudaFreeHost(b->h_e);
        b->d_clips = b->h_clips = nullptr;
        b->d_prefix = b->h_prefix = nullptr;
        b->d_e = b->h_e = nullptr;
        b->cap = 0;
        BCK(cudaMallocAsync((void **)&b->d_clips, sizeof(BatchClip) * cap, b->stream));
        BCK(cudaMallocHost((void **)&b->h_clips, sizeof(BatchClip) * cap));
        BCK(cudaMallocAsync((void **)&b->d_prefix, sizeof(int) * 3 * (cap + 1), b->stream));
        BCK(cudaMallocHost((void **)&b->h_prefix, sizeof(int) * 3 * (cap + 1)));
        BCK(cudaMallocAsync((void **)&b->d_e, sizeof(double) * cap, b->stream));
        BCK(cudaMallocHost((void **)&b->h_e, sizeof(double) * cap));
        b->cap = cap;
    }
    if (holes > b->change_cap) {
        long long cap = std::max(holes, 2 * b->change_cap);
        if (b->d_change) cudaFreeAsync(b->d_change, b->stream);
        b->d_change = nullptr;
        b->change_cap = 0;
        BCK(cudaMallocAsync((void **)&b->d_change, sizeof(float) * (size_t)std::max(cap, 1ll), b->stream));
        b->change_cap = cap;
    }
    if (chunks > b->chunks_cap) {
        const int cap = std::max(chunks, 2 * b->chunks_cap);
        if (b->d_chunks) cudaFreeAsync(b->d_chunks, b->stream);
        b->d_chunks = nullptr;
        b->chunks_cap = 0;
        BCK(cudaMallocAsync((void **)&b->d_chunks, sizeof(double) * (size_t)cap, b->stream));
        b->chunks_cap = cap;
    }
    return VI_OK;
}

// Moves a clip past the levels where it needs no more iterations (the loop
// condition of Algorithm 4: another iteration runs while e > stop and fewer
// than max_outer ran; e starts above any threshold), running the level
// transitions and the final step as vi_run does.
vi_status advance(vi_batch *b, Entry &c)
{
    while (c.state == CLIP_ITERATING) {
        const vi_config &cfg = c.ctx->cfg;
        const bool more = c.outer < cfg.max_outer && (c.outer == 0 || c.e > cfg.stop);
        if (more)
            return VI_OK;
        vi_status s;
        if (c.level > 0) {
            s = vi_next_level(c.ctx, c.level);
            c.level -= 1;
            c.outer = 0;
            c.e = INFINITY;
        } else {
            s = vi_final(c.ctx);
            c.state = CLIP_DONE;
        }
        if (s != VI_OK) {
            c.state = CLIP_FAILED;
            c.err = s;
            return bfail(b, s, std::string("clip ") + std::to_string(c.id) + ": " + vi_last_error(c.ctx));
        }
    }
    return VI_OK;
}

}  // namespace

extern "C" {

vi_status vi_batch_create(const vi_config *cfg, void *cuda_stream, vi_batch **out)
{
    if (!out)
        return VI_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return VI_ERR_NO_DEVICE;
    }
    vi_batch *b = new (std::nothrow) vi_batch();
    if (!b)
        return VI_ERR_OOM;
    if (cfg)
        b->cfg = *cfg;
    else
        vi_config_default(&b->cfg);
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return VI_ERR_CUDA;
        }
        b->own_stream = true;
    }
    if (cudaMallocAsync((void **)&b->counters, 6 * sizeof(unsigned long long), b->stream) != cudaSuccess) {
        vi_batch_destroy(b);
        return VI_ERR_OOM;
    }
    cudaMemsetAsync(b->counters, 0, 6 * sizeof(unsigned long long), b->stream);
    *out = b;
    return VI_OK;
}

void vi_batch_destroy(vi_batch *b)
{
    if (!b)
        return;
    if (b->stream)
        cudaStreamSynchronize(b->stream);
    for (Entry &c : b->clips)
        vi_ctx_destroy(c.ctx);
    if (b->d_clips) cudaFreeAsync(b->d_clips, b->stream);
    if (b->h_clips) cudaFreeHost(b->h_clips);
    if (b->d_prefix) cudaFreeAsync(b->d_prefix, b->stream);
    if (b->h_prefix) cudaFreeHost(b->h_prefix);
    if (b->d_e) cudaFreeAsync(b->d_e, b->stream);
    if (b->h_e) cudaFreeHost(b->h_e);
    if (b->d_change) cudaFreeAsync(b->d_change, b->stream);
    if (b->d_chunks) cudaFreeAsync(b->d_chunks, b->stream);
    if (b->counters) cudaFreeAsync(b->counters, b->stream);
    for (auto &e : b->events) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    if (b->own_stream && b->stream)
        cudaStreamDestroy(b->stream);
    delete b;
}

const char *vi_batch_last_error(const vi_batch *b) { return b ? b->err.c_str() : "null batch"; }

static vi_status vi_batch_add_body(vi_batch *b, const vi_config *job_cfg, const float *rgb, const uint8_t *mask, int W,
                       int H, int T, int ptr_is_device, int *id_out)
{
    if (!b || !id_out)
        return VI_ERR_ARG;
    vi_config cfg = job_cfg ? *job_cfg : b->cfg;
    if (cfg.use_texture != b->cfg.use_texture || cfg.n_pm != b->cfg.n_pm || cfg.storage != b->cfg.storage ||
        cfg.sub_sweeps != b->cfg.sub_sweeps)
        return bfail(b, VI_ERR_ARG, "vi_batch_add: use_texture, n_pm, sub_sweeps and storage must match the batch");
    vi_ctx *ctx = nullptr;
    vi_status s = vi_ctx_create(&cfg, b->stream, &ctx);
    if (s != VI_OK)
        return bfail(b, s, "vi_batch_add: context creation failed");
    s = vi_upload(ctx, rgb, mask, W, H, T, ptr_is_device);
    if (s == VI_OK)
        s = vi_prepare(ctx);
    if (s != VI_OK) {
        bfail(b, s, std::string("vi_batch_add: ") + vi_last_error(ctx));
        vi_ctx_destroy(ctx);
        return s;
    }
    Entry c;
    c.ctx = ctx;
    c.id = b->next_id++;
    c.level = ctx->L - 1;
    b->clips.push_back(c);
    *id_out = c.id;
    return advance(b, b->clips.back());
}

vi_status vi_batch_add(vi_batch *b, const vi_config *job_cfg, const float *rgb, const uint8_t *mask, int W,
                       int H, int T, int ptr_is_device, int *id_out)
{
    // host allocations proportional to the clip may throw; no exception crosses the C ABI
    try {
        return vi_batch_add_body(b, job_cfg, rgb, mask, W, H, T, ptr_is_device, id_out);
    } catch (...) {
        return VI_ERR_OOM;
    }
}

// Upload and preparation of one clip of vi_batch_add_many on its context's own
// stream, which first waits for everything the caller queued on the batch's
// stream before the call (ready), so that the inputs are complete.
static vi_status prepare_clip(vi_ctx *ctx, cudaEvent_t ready, int dev, const float *rgb, const uint8_t *mask, int W,
                              int H, int T, int ptr_is_device)
{
    if (cudaSetDevice(dev) != cudaSuccess || cudaStreamWaitEvent(ctx->stream, ready, 0) != cudaSuccess) {
        cudaGetLastError();
        return VI_ERR_CUDA;
    }
    vi_status s = vi_upload(ctx, rgb, mask, W, H, T, ptr_is_device);
    if (s == VI_OK)
        s = vi_prepare(ctx);
    if (s == VI_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        s = VI_ERR_CUDA;
    }
    return s;
}

static vi_status vi_batch_add_many_body(vi_batch *b, int n, const vi_config *const *job_cfgs,
                                        const float *const *rgbs, const uint8_t *const *masks, const int *Ws,
                                        const int *Hs, const int *Ts, int ptr_is_device, int n_threads,
                                        int *ids_out, vi_status *status_out)
{
    if (!b || n < 0 || (n > 0 && (!rgbs || !masks || !Ws || !Hs || !Ts || !ids_out)))
        return VI_ERR_ARG;
    if (n == 0)
        return VI_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, VI_ERR_NO_DEVICE, "vi_batch_add_many: no CUDA device");
    }
    std::vector<vi_ctx *> ctxs((size_t)n, nullptr);
    std::vector<vi_status> st((size_t)n, VI_OK);
    for (int i = 0; i < n; ++i) {
        ids_out[i] = -1;
        vi_config cfg = (job_cfgs && job_cfgs[i]) ? *job_cfgs[i] : b->cfg;
        if (cfg.use_texture != b->cfg.use_texture || cfg.n_pm != b->cfg.n_pm || cfg.storage != b->cfg.storage ||
            cfg.sub_sweeps != b->cfg.sub_sweeps) {
            st[(size_t)i] = VI_ERR_ARG;
            continue;
        }
        // a stream of its own for the preparation (priority from the clip's config)
        st[(size_t)i] = vi_ctx_create(&cfg, nullptr, &ctxs[(size_t)i]);
    }
    cudaEvent_t ready = nullptr;
    if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ready, b->stream) != cudaSuccess) {
        cudaGetLastError();
        for (vi_ctx *c : ctxs)
            vi_ctx_destroy(c);
        if (ready)
            cudaEventDestroy(ready);
        return bfail(b, VI_ERR_CUDA, "vi_batch_add_many: event");
    }
    // the clips' uploads and preparations run concurrently, one worker thread
    // each at a time: they are chains of small launches and synchronisations
    // that would otherwise leave the GPU idle between them
    std::atomic<int> next(0);
    auto work = [&]() {
        for (int i; (i = next.fetch_add(1)) < n;)
            if (st[(size_t)i] == VI_OK)
                st[(size_t)i] = prepare_clip(ctxs[(size_t)i], ready, dev, rgbs[i], masks[i], Ws[i], Hs[i], Ts[i],
                                             ptr_is_device);
    };
    const int nt = std::max(1, std::min(n, n_threads > 0 ? n_threads : 8));
    std::vector<std::thread> pool;
    try {
        for (int t = 1; t < nt; ++t)
            pool.emplace_back(work);
    } catch (...) {
        // fewer threads than asked for: the calling thread does the rest
    }
    work();
    for (std::thread &t : pool)
        t.join();
    cudaEventDestroy(ready);
    // the prepared clips join the batch's stream and its rounds, in order
    vi_status first = VI_OK;
    for (int i = 0; i < n; ++i) {
        vi_ctx *ctx = ctxs[(size_t)i];
        vi_status s = st[(size_t)i];
        if (s == VI_OK)
            s = ctx_adopt_stream(ctx, b->stream);
        if (s != VI_OK) {
            if (first == VI_OK) {
                first = s;
                bfail(b, s, "vi_batch_add_many: clip " + std::to_string(i) + ": " +
                                (ctx ? std::string(vi_last_error(ctx)) : std::string("bad configuration")));
            }
            vi_ctx_destroy(ctx);
            if (status_out)
                status_out[i] = s;
            continue;
        }
        Entry c;
        c.ctx = ctx;
        c.id = b->next_id++;
        c.level = ctx->L - 1;
        b->clips.push_back(c);
        ids_out[i] = c.id;
        s = advance(b, b->clips.back());
        if (status_out)
            status_out[i] = s;
        if (s != VI_OK && first == VI_OK)
            first = s;
    }
    return first;
}

vi_status vi_batch_add_many(vi_batch *b, int n, const vi_config *const *job_cfgs, const float *const *rgbs,
                            const uint8_t *const *masks, const int *Ws, const int *Hs, const int *Ts,
                            int ptr_is_device, int n_threads, int *ids_out, vi_status *status_out)
{
    try {
        return vi_batch_add_many_body(b, n, job_cfgs, rgbs, masks, Ws, Hs, Ts, ptr_is_device, n_threads, ids_out,
                                      status_out);
    } catch (...) {
        return VI_ERR_OOM;
    }
}

static vi_status vi_batch_step_body(vi_batch *b, int *n_active)
{
    const vi::Phase ph("batch round");
    if (!b)
        return VI_ERR_ARG;
    std::vector<Entry *> act;
    long long tot_t = 0, tot_h = 0, tot_c = 0;
    for (Entry &c : b->clips)
        if (c.state == CLIP_ITERATING)
            act.push_back(&c);
    const int n = (int)act.size();
    if (n > 0) {
        vi_status s = ensure_capacity(b, n, 0);
        if (s != VI_OK)
            return s;
        int *tpre_h = b->h_prefix, *hpre_h = b->h_prefix + b->cap + 1, *cpre_h = b->h_prefix + 2 * (b->cap + 1);
        for (int i = 0; i < n; ++i) {
            tpre_h[i] = (int)tot_t;
            hpre_h[i] = (int)tot_h;
            cpre_h[i] = (int)tot_c;
            // each clip's target range starts on a whole warp, so that a warp of
            // the step kernel holds targets of one clip (the kernels skip the padding)
            tot_t += (act[i]->ctx->lv[act[i]->level].nT + 31) & ~31;
            tot_h += act[i]->ctx->lv[act[i]->level].nH;
            tot_c += sum_chunks(act[i]->ctx->lv[act[i]->level].nH);
        }
        if (tot_t >= (1ll << 31) || tot_h >= (1ll << 31))
            return bfail(b, VI_ERR_ARG, "vi_batch_step: batch larger than 2^31 targets");
        tpre_h[n] = (int)tot_t;
        hpre_h[n] = (int)tot_h;
        cpre_h[n] = (int)tot_c;
        s = ensure_capacity(b, n, tot_h, (int)std::max(tot_c, 1ll));
        if (s != VI_OK)
            return s;
        const int c5 = b->cfg.use_texture != 0;
        for (int i = 0; i < n; ++i) {
            vi_ctx *ctx = act[i]->ctx;
            const int level = act[i]->level;
            Level &l = ctx->lv[level];
            BatchClip &bc = b->h_clips[i];
            AnnArgs a;
            std::memset(&a, 0, sizeof(a));
            a.L = l.view();   // h4 set only at a level the search screens (screen_level)
            a.targets = l.targets;
            a.nT = l.nT;
            a.tmask = l.code;
            a.tbit = CODE_TARGET;
            a.excl = nullptr;
            a.rmax = std::max(l.W, std::max(l.H, l.T));
            a.rho_log2 = ctx->rho_log2;
            a.key0 = (uint32_t)(ctx->cfg.seed & 0xFFFFFFFFull);
            a.key1 = (uint32_t)(ctx->cfg.seed >> 32);
            a.tag = make_tag(PURPOSE_SEARCH, level, act[i]->outer);
            a.clip = ctx->cfg.clip;
            a.rs_mode = ctx->cfg.rs_mode;
            a.do_random = 1;
            a.chg_span = 0;     // the batch step kernel sets the span from k
            a.phi_in = l.phi[0];
            a.d_in = l.d2[0];
            a.phi_out = l.phi[1];
            a.d_out = l.d2[1];
            a.chg_in = l.chg[0];
            a.chg_out = l.chg[1];
            bc.odd = a;
            a.phi_in = l.phi[1];
            a.d_in = l.d2[1];
            a.phi_out = l.phi[0];
            a.d_out = l.d2[0];
            a.chg_in = l.chg[1];
            a.chg_out = l.chg[0];
            bc.even = a;
            VoteArgs v;
            v.L = l.view();
            v.list = l.holes;
            v.n = l.nH;
            v.phi = l.phi[0];
            v.d2 = l.d2[0];
            // every patch covering a voxel of H is centred in H~ (the 5x5x5 dilation
            // of H), so the vote needs no per-patch set test
            v.allowed = nullptr;
            v.abit = CODE_TARGET;
            v.weighted = ctx->cfg.weighted;
            v.hp = nullptr;
            v.partials = b->d_change + b->h_prefix[b->cap + 1 + i];
            bc.vote = v;
            bc.d0 = l.d2[0];
        }
        cudaStream_t st = b->stream;
        BCK(cudaMemcpyAsync(b->d_clips, b->h_clips, sizeof(BatchClip) * n, cudaMemcpyHostToDevice, st));
        BCK(cudaMemcpyAsync(b->d_prefix, b->h_prefix, sizeof(int) * 3 * (b->cap + 1), cudaMemcpyHostToDevice,
                            st));
        const int *tpre = b->d_prefix, *hpre = b->d_prefix + b->cap + 1, *cpre = b->d_prefix + 2 * (b->cap + 1);
        // the warp-shared form (32) exists for the step; the rescore then uses one lane per target
        const int lanes = b->cfg.lanes_per_target;
        const int rescore_lanes = lanes == 32 ? 1 : lanes;
        launch_rescore_batch(b->d_clips, tpre, n, (int)tot_t, c5, b->counters, rescore_lanes, st);
        const int J = std::max(b->cfg.sub_sweeps, 1);
        int sweep = 0;
        for (int k = 1; k <= b->cfg.n_pm; ++k)
            for (int j = 0; j < J; ++j, ++sweep) {
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (b->profiling) {
                if (b->events_used == b->events.size()) {
                    cudaEvent_t x, y;
                    BCK(cudaEventCreate(&x));
                    BCK(cudaEventCreate(&y));
                    b->events.emplace_back(x, y);
                }
                e0 = b->events[b->events_used].first;
                e1 = b->events[b->events_used].second;
                ++b->events_used;
                BCK(cudaEventRecord(e0, st));
            }
            // the span of vi_run's sweeps: the previous sub-sweep, or at the
            // first sub-sweep of iteration k >= 3 the last of iteration k - 2
            BatchSweep w;
            w.k = k;
            w.sweep = sweep;
            w.span = j > 0 ? 1 : (k >= 3 && J + 1 <= 8 ? J + 1 : 0);
            w.do_random = j == J - 1;
            launch_ann_step_batch(b->d_clips, tpre, n, (int)tot_t, w, c5, b->cfg.storage != 0, b->counters + 1,
                                  lanes, st);
            if (b->profiling)
                BCK(cudaEventRecord(e1, st));
        }
        if (sweep & 1)
            for (int i = 0; i < n; ++i) {
                Level &l = act[i]->ctx->lv[act[i]->level];
                launch_copy_targets(l.targets, l.nT, l.phi[1], l.d2[1], l.phi[0], l.d2[0], st);
            }
        launch_vote_batch(b->d_clips, hpre, n, (int)tot_h, c5, st);
        launch_segment_sums(b->d_change, hpre, cpre, n, (int)tot_c, b->d_chunks, b->d_e, st);
        BCK(cudaGetLastError());
        BCK(cudaMemcpyAsync(b->h_e, b->d_e, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        BCK(cudaStreamSynchronize(st));
        ++b->rounds;
        for (int i = 0; i < n; ++i) {
            Entry &c = *act[i];
            const int nH = c.ctx->lv[c.level].nH;
            c.e = nH ? (float)(b->h_e[i] / (3.0 * nH)) : 0.0f;
            c.outer += 1;
            if (c.level < 16)
                c.ctx->outer[c.level] += 1;
            vi_status s2 = advance(b, c);
            if (s2 != VI_OK)
                return s2;
        }
    }
    if (n_active) {
        int m = 0;
        for (Entry &c : b->clips)
            m += c.state == CLIP_ITERATING;
        *n_active = m;
    }
    return VI_OK;
}

vi_status vi_batch_step(vi_batch *b, int *n_active)
{
    // host allocations proportional to the clip may throw; no exception crosses the C ABI
    try {
        return vi_batch_step_body(b, n_active);
    } catch (...) {
        return VI_ERR_OOM;
    }
}

vi_status vi_batch_run(vi_batch *b)
{
    if (!b)
        return VI_ERR_ARG;
    int active = 1;
    while (active > 0) {
        vi_status s = vi_batch_step(b, &active);
        if (s != VI_OK)
            return s;
    }
    return VI_OK;
}

vi_status vi_batch_poll(vi_batch *b, int id, int *done, int *level)
{
    if (!b)
        return VI_ERR_ARG;
    Entry *c = find(b, id);
    if (!c)
        return bfail(b, VI_ERR_ARG, "vi_batch_poll: unknown clip");
    if (done)
        *done = c->state == CLIP_DONE ? 1 : (c->state == CLIP_FAILED ? -1 : 0);
    if (level)
        *level = c->level;
    return VI_OK;
}

vi_status vi_batch_fetch(vi_batch *b, int id, float *rgb_out, int ptr_is_device)
{
    if (!b || !rgb_out)
        return VI_ERR_ARG;
    Entry *c = find(b, id);
    if (!c)
        return bfail(b, VI_ERR_ARG, "vi_batch_fetch: unknown clip");
    if (c->state != CLIP_DONE)
        return bfail(b, VI_ERR_STATE, "vi_batch_fetch: clip not finished");
    vi_status s = vi_fetch_result(c->ctx, rgb_out, ptr_is_device);
    if (s != VI_OK)
        return bfail(b, s, vi_last_error(c->ctx));
    return VI_OK;
}

vi_status vi_batch_remove(vi_batch *b, int id)
{
    if (!b)
        return VI_ERR_ARG;
    for (size_t i = 0; i < b->clips.size(); ++i)
        if (b->clips[i].id == id) {
            vi_stats s;
            if (vi_get_stats(b->clips[i].ctx, &s) == VI_OK)
                b->removed_evals += s.evals;
            vi_ctx_destroy(b->clips[i].ctx);
            b->clips.erase(b->clips.begin() + (long)i);
            return VI_OK;
        }
    return bfail(b, VI_ERR_ARG, "vi_batch_remove: unknown clip");
}

vi_status vi_batch_clip_stats(vi_batch *b, int id, vi_stats *out)
{
    if (!b || !out)
        return VI_ERR_ARG;
    Entry *c = find(b, id);
    if (!c)
        return bfail(b, VI_ERR_ARG, "vi_batch_clip_stats: unknown clip");
    return vi_get_stats(c->ctx, out);
}

vi_status vi_batch_clip_ctx(vi_batch *b, int id, vi_ctx **ctx_out, int *call_out)
{
    if (!b || !ctx_out)
        return VI_ERR_ARG;
    Entry *c = find(b, id);
    if (!c)
        return bfail(b, VI_ERR_ARG, "vi_batch_clip_ctx: unknown clip");
    *ctx_out = c->ctx;
    if (call_out)
        *call_out = c->outer;
    return VI_OK;
}

vi_status vi_batch_profile(vi_batch *b, int enable)
{
    if (!b)
        return VI_ERR_ARG;
    b->profiling = enable != 0;
    return VI_OK;
}

vi_status vi_batch_step_time(vi_batch *b, double *step_ms, unsigned long long *step_evals)
{
    if (!b)
        return VI_ERR_ARG;
    unsigned long long h[3] = {0, 0, 0};
    BCK(cudaMemcpyAsync(h, b->counters, sizeof(h), cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    for (size_t i = 0; i < b->events_used; ++i) {
        float ms = 0.0f;
        BCK(cudaEventElapsedTime(&ms, b->events[i].first, b->events[i].second));
        b->step_ms += ms;
    }
    b->events_used = 0;
    if (step_ms)
        *step_ms = b->step_ms;
    if (step_evals)
        *step_evals = h[1];
    return VI_OK;
}

vi_status vi_batch_get_stats(vi_batch *b, unsigned long long *evals, unsigned long long *gathered,
                             unsigned long long *rounds)
{
    if (!b)
        return VI_ERR_ARG;
    unsigned long long h[3] = {0, 0, 0};
    BCK(cudaMemcpyAsync(h, b->counters, sizeof(h), cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    unsigned long long ev = h[0] + h[1] + b->removed_evals;
    for (Entry &c : b->clips) {
        vi_stats s;
        if (vi_get_stats(c.ctx, &s) == VI_OK)
            ev += s.evals;   // the clip's own launches: preparation, transitions
    }
    if (evals)
        *evals = ev;
    if (gathered)
        *gathered = h[2];
    if (rounds)
        *rounds = b->rounds;
    return VI_OK;
}

vi_status vi_batch_screen_stats(vi_batch *b, unsigned long long *gathered_h, unsigned long long *screened,
                                unsigned long long *passed)
{
    if (!b)
        return VI_ERR_ARG;
    unsigned long long h[6] = {0, 0, 0, 0, 0, 0};
    BCK(cudaMemcpyAsync(h, b->counters, sizeof(h), cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    if (gathered_h)
        *gathered_h = h[3];
    if (screened)
        *screened = h[4];
    if (passed)
        *passed = h[5];
    return VI_OK;
}

}  // extern "C"
