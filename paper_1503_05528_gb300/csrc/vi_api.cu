// vi_api.cu -- host runtime and C ABI of the library (declared in vi.h).
//
// A context owns one clip: its input copy, the per-level device buffers of the
// pyramid (channels, set codes, voxel lists, two shift/distance buffers for the
// Jacobi sweeps) and the scratch of the reductions. Every kernel is launched on
// the context's stream; host synchronisation happens only where a value must
// come back (list sizes after the pyramid, the stopping criterion, onion-peel
// layer sizes, fetches).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "vi_ctx.h"

using namespace vi;

std::atomic<unsigned long long> vi::g_launch_count{0};

vi_status vi::ctx_fail(vi_ctx *ctx, vi_status st, const std::string &msg)
{
    if (ctx)
        ctx->err = msg;
    return st;
}

namespace {

vi_status fail(vi_ctx *ctx, vi_status st, const std::string &msg)
{
    if (ctx)
        ctx->err = msg;
    return st;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(ctx, VI_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
    } while (0)

#define CK_LAUNCH()                                                                               \
    do {                                                                                          \
        cudaError_t e_ = cudaGetLastError();                                                      \
        if (e_ != cudaSuccess)                                                                    \
            return fail(ctx, VI_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
    } while (0)

#define TRY(expr)                                                                                 \
    do {                                                                                          \
        vi_status s_ = (expr);                                                                    \
        if (s_ != VI_OK)                                                                          \
            return s_;                                                                            \
    } while (0)

// Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the
// context's stream, from the device's default pool): allocating and freeing
// never synchronises the device, so contexts on other streams keep running
// while one is created, re-uploaded or destroyed.
template <typename P>
vi_status dalloc(vi_ctx *ctx, P **ptr, size_t bytes)
{
    *ptr = nullptr;
    if (bytes == 0)
        bytes = 16;
    if (ctx->cfg.mem_limit && ctx->held + bytes > ctx->cfg.mem_limit)
        return fail(ctx, VI_ERR_OOM,
                    "allocation of " + std::to_string(bytes) + " bytes beyond the context's memory limit (" +
                        std::to_string(ctx->held) + " of " + std::to_string(ctx->cfg.mem_limit) + " held)");
    cudaError_t e = cudaMallocAsync((void **)ptr, bytes, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return fail(ctx, e == cudaErrorMemoryAllocation ? VI_ERR_OOM : VI_ERR_CUDA,
                    std::string("cudaMallocAsync(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    try {
        ctx->sizes[(const void *)*ptr] = bytes;
    } catch (...) {
        cudaFreeAsync((void *)*ptr, ctx->stream);
        *ptr = nullptr;
        return fail(ctx, VI_ERR_OOM, "host allocation");
    }
    ctx->held += bytes;
    return VI_OK;
}

template <typename P>
void dfree(vi_ctx *ctx, P *&ptr)
{
    if (ptr) {
        auto it = ctx->sizes.find((const void *)ptr);
        if (it != ctx->sizes.end()) {
            ctx->held -= it->second;
            ctx->sizes.erase(it);
        }
        cudaFreeAsync((void *)ptr, ctx->stream);
    }
    ptr = nullptr;
}

// The default pool of each device keeps freed memory for the next
// allocation instead of returning it at every synchronisation (set once per
// device and process).
void keep_pool_memory()
{
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev])
        return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done[dev] = true;
}

void free_state(vi_ctx *ctx)
{
    if (ctx->stream)
        cudaStreamSynchronize(ctx->stream);
    for (Level &l : ctx->lv) {
        dfree(ctx, l.x4);
        dfree(ctx, l.x1);
        dfree(ctx, l.code);
        dfree(ctx, l.h4);
        dfree(ctx, l.hmax);
        dfree(ctx, l.phi[0]);
        dfree(ctx, l.phi[1]);
        dfree(ctx, l.d2[0]);
        dfree(ctx, l.d2[1]);
        dfree(ctx, l.chg[0]);
        dfree(ctx, l.chg[1]);
        dfree(ctx, l.targets);
        dfree(ctx, l.holes);
        dfree(ctx, l.sources);
    }
    ctx->lv.clear();
    dfree(ctx, ctx->rgb);
    dfree(ctx, ctx->mask);
    dfree(ctx, ctx->out_rgb);
    dfree(ctx, ctx->T0);
    dfree(ctx, ctx->tmpA);
    dfree(ctx, ctx->tmpB);
    dfree(ctx, ctx->block_counts);
    dfree(ctx, ctx->partials);
    dfree(ctx, ctx->partials2);
    dfree(ctx, ctx->chunks);
    dfree(ctx, ctx->hp);
    dfree(ctx, ctx->layer);
    dfree(ctx, ctx->ltgt);
    dfree(ctx, ctx->layer_list);
    dfree(ctx, ctx->ltgt_list);
    ctx->partials_cap = ctx->partials2_cap = ctx->chunks_cap = 0;
    ctx->uploaded = ctx->built = false;
}

vi_status check_config(vi_ctx *ctx, const vi_config *c)
{
    if (!(c->lambda >= 0.0f) || c->n_pm < 0 || c->n_pm > 255 || c->levels < 0 || c->levels > 15 ||
        c->rs_mode < 0 || c->rs_mode > 1 || c->sub_sweeps < 1 || c->sub_sweeps > 16 ||
        c->time_subsample < 0 || c->time_subsample > 1 ||
        c->max_outer < 0 || c->max_outer > 65535 || !(c->stop >= 0.0f) || (c->storage < 0 || c->storage > 2) ||
        !(c->lanes_per_target == 0 || c->lanes_per_target == 1 || c->lanes_per_target == 2 ||
          c->lanes_per_target == 4 || c->lanes_per_target == 8 || c->lanes_per_target == 32))
        return fail(ctx, VI_ERR_ARG, "invalid vi_config field");
    // rho must be 2^-m, m >= 1
    int m = 0;
    float r = c->rho;
    while (r < 1.0f && r > 0.0f && m < 30) {
        r *= 2.0f;
        ++m;
    }
    if (!(r == 1.0f) || m < 1)
        return fail(ctx, VI_ERR_ARG, "rho must be 1/2^m with m >= 1");
    ctx->rho_log2 = m;
    return VI_OK;
}

bool level_ok(vi_ctx *ctx, int level) { return ctx->built && level >= 0 && level < ctx->L; }

vi_status ensure_partials(vi_ctx *ctx, int n_blocks)
{
    if (n_blocks <= ctx->partials_cap)
        return VI_OK;
    dfree(ctx, ctx->partials);
    TRY(dalloc(ctx, &ctx->partials, sizeof(float) * (size_t)n_blocks));
    ctx->partials_cap = n_blocks;
    return VI_OK;
}

vi_status ensure_partials2(vi_ctx *ctx, int n_blocks)
{
    if (n_blocks <= ctx->partials2_cap)
        return VI_OK;
    dfree(ctx, ctx->partials2);
    TRY(dalloc(ctx, &ctx->partials2, 2 * sizeof(double) * (size_t)n_blocks));
    ctx->partials2_cap = n_blocks;
    return VI_OK;
}

// Lanes per target of the rescore kernels: the warp-shared form (32) exists
// for the step only; the rescore then uses one lane per target.
static int rescore_lanes(int lanes) { return lanes == 32 ? 1 : lanes; }

// One launch of the PatchMatch step kernel.
vi_status step_launch(vi_ctx *ctx, const AnnArgs &a)
{
    launch_ann_step(a, ctx->c5, ctx->stream);
    CK_LAUNCH();
    ++ctx->step_launches;
    return VI_OK;
}

// With profiling on, an event pair around a run of back-to-back step launches.
vi_status profile_begin(vi_ctx *ctx, cudaEvent_t *e1)
{
    *e1 = nullptr;
    if (!ctx->profiling)
        return VI_OK;
    if (ctx->events_used == ctx->events.size()) {
        cudaEvent_t x, y;
        CK(cudaEventCreate(&x));
        CK(cudaEventCreate(&y));
        ctx->events.emplace_back(x, y);
        ctx->event_launches.push_back(0);
    }
    CK(cudaEventRecord(ctx->events[ctx->events_used].first, ctx->stream));
    *e1 = ctx->events[ctx->events_used].second;
    return VI_OK;
}

vi_status profile_end(vi_ctx *ctx, cudaEvent_t e1, int launches)
{
    if (!e1)
        return VI_OK;
    CK(cudaEventRecord(e1, ctx->stream));
    ctx->event_launches[ctx->events_used] = launches;
    ++ctx->events_used;
    return VI_OK;
}

// The arguments of sweep s of a search over a target list: iteration k,
// sub-sweep j; sweep s reads buffer s & 1 and writes the other one.
AnnArgs sweep_args(vi_ctx *ctx, int level, const int *targets, int nT, const uint8_t *tmask, uint8_t tbit,
                   const uint8_t *excl, uint32_t tag, int k, int j, int s)
{
    Level &l = ctx->lv[level];
    AnnArgs a;
    a.L = l.view();   // h4 set only at a level the search screens (screen_level)
    a.targets = targets;
    a.nT = nT;
    a.phi_in = l.phi[s & 1];
    a.d_in = l.d2[s & 1];
    a.phi_out = l.phi[(s + 1) & 1];
    a.d_out = l.d2[(s + 1) & 1];
    a.tmask = tmask;
    a.tbit = tbit;
    a.excl = excl;
    a.k = k;
    a.rmax = std::max(l.W, std::max(l.H, l.T));
    a.rho_log2 = ctx->rho_log2;
    a.key0 = (uint32_t)(ctx->cfg.seed & 0xFFFFFFFFull);
    a.key1 = (uint32_t)(ctx->cfg.seed >> 32);
    a.tag = tag;
    a.clip = ctx->cfg.clip;
    a.evals = ctx->evals_dev + 1;
    a.gathered = ctx->evals_dev + 2;
    a.screen = ctx->evals_dev + 3;
    a.lanes = ctx->cfg.lanes_per_target;
    a.rs_mode = ctx->cfg.rs_mode;
    a.do_random = j == ctx->cfg.sub_sweeps - 1;
    // sweeps since the same targets judged the same neighbours in the same
    // direction: the previous sub-sweep, or at the first sub-sweep of
    // iteration k >= 3 the last of iteration k - 2
    const int J = ctx->cfg.sub_sweeps;
    int span = 0;
    if (j > 0)
        span = 1;
    else if (k >= 3 && J + 1 <= 8)
        span = J + 1;
    a.chg_in = l.chg[s & 1];
    a.chg_out = l.chg[(s + 1) & 1];
    a.chg_span = span;
    return a;
}

// Distances, then n_pm Jacobi sweeps (Algorithm 1) over a target list. The
// current shift map is buffer 0; sweep k reads buffer (k-1)&1 and writes k&1,
// so only target entries are ever read from buffer 1; after an odd count the
// targets are copied back to buffer 0.
vi_status run_ann(vi_ctx *ctx, int level, const int *targets, int nT, const uint8_t *tmask,
                  uint8_t tbit, const uint8_t *excl, uint32_t tag)
{
    const Phase ph("search L%d", level);
    Level &l = ctx->lv[level];
    launch_rescore(l.view(), targets, nT, l.phi[0], l.d2[0], excl, ctx->c5, ctx->evals_dev, ctx->stream,
                   rescore_lanes(ctx->cfg.lanes_per_target));
    CK_LAUNCH();
    cudaEvent_t e1 = nullptr;
    TRY(profile_begin(ctx, &e1));
    int s = 0;
    for (int k = 1; k <= ctx->cfg.n_pm; ++k)
        for (int j = 0; j < ctx->cfg.sub_sweeps; ++j, ++s)
            TRY(step_launch(ctx, sweep_args(ctx, level, targets, nT, tmask, tbit, excl, tag, k, j, s)));
    TRY(profile_end(ctx, e1, s));
    if (s & 1) {
        launch_copy_targets(targets, nT, l.phi[1], l.d2[1], l.phi[0], l.d2[0], ctx->stream);
        CK_LAUNCH();
    }
    return VI_OK;
}

// The vote of the occluded voxels [off, off + n) of the level's list; their
// changes go to partials[off .. off + n).
vi_status vote_range(vi_ctx *ctx, int level, int off, int n)
{
    Level &l = ctx->lv[level];
    TRY(ensure_partials(ctx, std::max(l.nH, 1)));
    VoteArgs a;
    a.L = l.view();
    a.list = l.holes + off;
    a.n = n;
    a.phi = l.phi[0];
    a.d2 = l.d2[0];
    // every patch covering a voxel of H is centred in H~ (the 5x5x5 dilation
    // of H), so the vote needs no per-patch set test
    a.allowed = nullptr;
    a.abit = CODE_TARGET;
    a.weighted = ctx->cfg.weighted;
    a.hp = nullptr;
    a.partials = ctx->partials + off;
    launch_vote(a, ctx->c5, ctx->stream);
    CK_LAUNCH();
    return VI_OK;
}

// e's numerator of Sec. 3.7 (the per-voxel changes of the whole list summed
// in the fixed two-stage order) into change_dev.
vi_status sum_changes(vi_ctx *ctx, int level, double *change_dev)
{
    const int nH = ctx->lv[level].nH;
    const int nc = std::max(sum_chunks(nH), 1);
    if (nc > ctx->chunks_cap) {
        dfree(ctx, ctx->chunks);
        ctx->chunks_cap = 0;
        TRY(dalloc(ctx, &ctx->chunks, sizeof(double) * (size_t)nc));
        ctx->chunks_cap = nc;
    }
    launch_sum_partials(ctx->partials, nH, ctx->chunks, change_dev, ctx->stream);
    CK_LAUNCH();
    return VI_OK;
}

vi_status vote_level(vi_ctx *ctx, int level, double *change_dev)
{
    const Phase ph("vote L%d", level);
    TRY(vote_range(ctx, level, 0, ctx->lv[level].nH));
    if (change_dev)
        TRY(sum_changes(ctx, level, change_dev));
    return VI_OK;
}

}  // namespace

vi_status vi::ctx_ensure_partials(vi_ctx *ctx, int n) { return ensure_partials(ctx, n); }

bool vi::screen_level(const vi_ctx *ctx, const Level &l)
{
    if (ctx->cfg.storage == 2)
        return true;
    if (ctx->cfg.storage != 1)
        return false;
    static long long l2 = -1;
    if (l2 < 0) {
        int dev = 0, bytes = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&bytes, cudaDevAttrL2CacheSize, dev) != cudaSuccess || bytes <= 0) {
            cudaGetLastError();
            bytes = 128 << 20;
        }
        l2 = bytes;
    }
    const long long channel_bytes = (long long)l.V * (ctx->c5 ? 20 : 16);
    return channel_bytes > l2;
}

vi_status vi::ctx_adopt_stream(vi_ctx *ctx, cudaStream_t st)
{
    if (!ctx)
        return VI_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->own_stream && ctx->stream)
        CK(cudaStreamDestroy(ctx->stream));
    ctx->stream = st;
    ctx->own_stream = false;
    return VI_OK;
}

namespace {

// The level rule of Sec. 3.6 for the largest per-frame extent of the hole: the
// smallest L with ext / 2^(L-1) <= 9, keeping the next level's side >= 16.
int levels_for_extent(int ext, int W, int H)
{
    int L = 1;
    while (true) {
        const int scale = 1 << (L - 1);
        if ((ext + scale - 1) / scale <= 9)
            break;
        const int side = (std::min(W, H) + 2 * scale - 1) / (2 * scale);   // next level's side
        if (side < 16 || L >= 15)
            break;
        ++L;
    }
    return L;
}

int host_auto_levels(const uint8_t *mask, int W, int H, int T)
{
    int ext = 0;
    for (int t = 0; t < T; ++t) {
        int x0 = W, x1 = -1, y0 = H, y1 = -1;
        const uint8_t *m = mask + (size_t)t * W * H;
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x)
                if (m[(size_t)y * W + x]) {
                    x0 = std::min(x0, x);
                    x1 = std::max(x1, x);
                    y0 = std::min(y0, y);
                    y1 = std::max(y1, y);
                }
        if (x1 >= 0)
            ext = std::max(ext, std::max(x1 - x0 + 1, y1 - y0 + 1));
    }
    return levels_for_extent(ext, W, H);
}

}  // namespace

extern "C" {

void vi_config_default(vi_config *cfg)
{
    if (!cfg)
        return;
    cfg->lambda = 50.0f;
    cfg->n_pm = 10;
    cfg->rho = 0.5f;
    cfg->levels = 0;
    cfg->max_outer = 20;
    cfg->stop = 0.1f / 255.0f;
    cfg->weighted = 1;
    cfg->use_texture = 1;
    cfg->storage = 0;
    cfg->seed = 1503;
    cfg->clip = 0;
    cfg->lanes_per_target = 0;
    cfg->stream_priority = 0;
    cfg->rs_mode = 0;
    cfg->sub_sweeps = 2;
    cfg->time_subsample = 0;
    cfg->mem_limit = 0;
}

vi_status vi_ctx_create(const vi_config *cfg, void *cuda_stream, vi_ctx **out)
{
    if (!out)
        return VI_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return VI_ERR_NO_DEVICE;
    }
    vi_ctx *ctx = new (std::nothrow) vi_ctx();
    if (!ctx)
        return VI_ERR_OOM;
    if (cfg)
        ctx->cfg = *cfg;
    else
        vi_config_default(&ctx->cfg);
    vi_status s = check_config(ctx, &ctx->cfg);
    if (s != VI_OK) {
        delete ctx;
        return s;
    }
    ctx->c5 = ctx->cfg.use_texture != 0;
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        const int prio = std::min(least, std::max(greatest, ctx->cfg.stream_priority));
        if (cudaStreamCreateWithPriority(&ctx->stream, cudaStreamNonBlocking, prio) != cudaSuccess) {
            cudaGetLastError();
            delete ctx;
            return VI_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    keep_pool_memory();
    if (dalloc(ctx, &ctx->count_dev, 64 * sizeof(int)) != VI_OK ||
        dalloc(ctx, &ctx->scal, 8 * sizeof(double)) != VI_OK ||
        dalloc(ctx, &ctx->evals_dev, 6 * sizeof(unsigned long long)) != VI_OK) {
        vi_ctx_destroy(ctx);
        return VI_ERR_OOM;
    }
    cudaMemsetAsync(ctx->evals_dev, 0, 6 * sizeof(unsigned long long), ctx->stream);
    *out = ctx;
    return VI_OK;
}

void vi_ctx_destroy(vi_ctx *ctx)
{
    if (!ctx)
        return;
    free_state(ctx);
    dfree(ctx, ctx->count_dev);
    dfree(ctx, ctx->scal);
    dfree(ctx, ctx->evals_dev);
    for (auto &e : ctx->events) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    if (ctx->own_stream && ctx->stream)
        cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char *vi_last_error(const vi_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int vi_auto_levels(const uint8_t *mask_host, int W, int H, int T)
{
    if (!mask_host || W <= 0 || H <= 0 || T <= 0)
        return 1;
    return host_auto_levels(mask_host, W, H, T);
}

size_t vi_footprint_bytes(const vi_config *cfg, int W, int H, int T, long long hole_voxels)
{
    (void)hole_voxels;
    const int L = (cfg && cfg->levels > 0) ? cfg->levels : 6;
    const bool c5 = !cfg || cfg->use_texture;
    size_t total = 0;
    int w = W, h = H;
    for (int l = 0; l < L; ++l) {
        const size_t V = (size_t)w * h * T;
        // x4, x1, code, 2 shift + 2 distance + 2 change-flag buffers, three lists (upper bound),
        // FP16 copies
        total += V * (16 + (c5 ? 4 : 0) + 1 + 16 + 8 + 2 + 12);
        if (cfg && cfg->storage != 0)
            total += V * 8 + 256;
        w = (w + 1) / 2;
        h = (h + 1) / 2;
    }
    const size_t V0 = (size_t)W * H * T;
    total += V0 * (12 + 1 + 2 + (c5 ? 8 + 8 + 1 + 8 + 4 : 0));
    return total + (16u << 20);
}

// The device address of host memory registered with CUDA (pinned: cudaHostAlloc,
// cudaMallocHost, cudaHostRegister), or nullptr for other memory. Copies to
// and from registered host memory run as kernels through that address: after
// the GPU has worked on its own memory for a while, the copy engine's first
// pass over the host pages is slow (measured on GB300: 57 ms to fetch 1.96 GB
// into pinned buffers after a 48-clip batch, 5 ms from device to device).
static void *mapped_host_byte(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// The device address of a registered host buffer of `bytes` bytes, when its
// first and its last byte are both registered and map to addresses `bytes - 1`
// apart; nullptr otherwise (the copy engine then moves it).
static void *mapped_host(const void *p, size_t bytes)
{
    void *d = mapped_host_byte(p);
    if (!d || bytes == 0)
        return d;
    const void *last = static_cast<const char *>(p) + (bytes - 1);
    void *dl = mapped_host_byte(last);
    return dl == static_cast<char *>(d) + (bytes - 1) ? d : nullptr;
}

// bytes from a caller's buffer (device memory, or host memory) into dst.
static cudaError_t copy_in(void *dst, const void *src, size_t bytes, int ptr_is_device, cudaStream_t st)
{
    if (!ptr_is_device) {
        if (const void *mapped = mapped_host(src, bytes)) {
            launch_copy_bytes(dst, mapped, (long long)bytes, st);
            return cudaGetLastError();
        }
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
    }
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st);
}

static vi_status vi_upload_body(vi_ctx *ctx, const float *rgb, const uint8_t *mask, int W, int H, int T,
                    int ptr_is_device)
{
    if (!ctx)
        return VI_ERR_ARG;
    if (!rgb || !mask || W <= 0 || H <= 0 || T <= 0 || W > 32767 || H > 32767 || T > 32767 ||
        (long long)W * H * T >= (1ll << 31))
        return fail(ctx, VI_ERR_ARG, "vi_upload: bad pointer or size");
    free_state(ctx);
    ctx->W = W;
    ctx->H = H;
    ctx->T = T;
    ctx->V0 = W * H * T;
    const size_t V0 = (size_t)ctx->V0;

    TRY(dalloc(ctx, &ctx->rgb, V0 * 3 * sizeof(float)));
    TRY(dalloc(ctx, &ctx->mask, V0));
    CK(copy_in(ctx->rgb, rgb, V0 * 3 * sizeof(float), ptr_is_device, ctx->stream));
    CK(copy_in(ctx->mask, mask, V0, ptr_is_device, ctx->stream));
    if (!ptr_is_device)
        CK(cudaStreamSynchronize(ctx->stream));   // the caller may reuse its host buffers on return

    int L = ctx->cfg.levels;
    if (L <= 0) {
        // the level rule from the hole's per-frame extents, found on the
        // device (16 bytes per frame come back) instead of a scan of the mask
        // on the host
        int4 *ext_dev = nullptr;
        TRY(dalloc(ctx, &ext_dev, sizeof(int4) * (size_t)T));
        std::vector<int4> ext_host((size_t)T);
        launch_mask_extents(ctx->mask, W, H, T, ext_dev, ctx->stream);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ext_host.data(), ext_dev, sizeof(int4) * (size_t)T, cudaMemcpyDeviceToHost,
                                ctx->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(ctx->stream);
        dfree(ctx, ext_dev);
        if (e != cudaSuccess)
            return fail(ctx, VI_ERR_CUDA, std::string("vi_upload: ") + cudaGetErrorString(e));
        int ext = 0;
        for (const int4 &f : ext_host)
            if (f.y >= 0)
                ext = std::max(ext, std::max(f.y - f.x + 1, f.w - f.z + 1));
        L = levels_for_extent(ext, W, H);
    }
    ctx->L = L;
    TRY(dalloc(ctx, &ctx->tmpA, V0));
    TRY(dalloc(ctx, &ctx->tmpB, V0));
    {
        // the per-block counts of every level's three lists (kept from the
        // sizing pass to the writing pass), or of one level-0 list
        size_t n = 0;
        int w = W, h = H, tl = T;
        for (int l = 0; l < L; ++l) {
            n += 3 * (size_t)(compact_blocks(w * h * tl) + 1);
            w = (w + 1) / 2;
            h = (h + 1) / 2;
            if (ctx->cfg.time_subsample)
                tl = (tl + 1) / 2;
        }
        n = std::max(n, (size_t)compact_blocks(ctx->V0) + 1);
        TRY(dalloc(ctx, &ctx->block_counts, sizeof(int) * n));
    }

    ctx->lv.assign(L, Level());
    int w = W, h = H, tl = T;
    for (int l = 0; l < L; ++l) {
        Level &lv = ctx->lv[l];
        lv.W = w;
        lv.H = h;
        lv.T = tl;
        lv.V = w * h * tl;
        const size_t V = (size_t)lv.V;
        TRY(dalloc(ctx, &lv.x4, V * sizeof(float4)));
        if (ctx->c5)
            TRY(dalloc(ctx, &lv.x1, V * sizeof(float)));
        TRY(dalloc(ctx, &lv.code, V));
        if (screen_level(ctx, lv)) {
            // FP16 copies only where the search screens with them: a level
            // that is never screened needs neither the copy nor its upkeep
            TRY(dalloc(ctx, &lv.h4, V * sizeof(uint2)));
            TRY(dalloc(ctx, &lv.hmax, 8 * sizeof(unsigned)));
        }
        for (int b = 0; b < 2; ++b) {
            TRY(dalloc(ctx, &lv.phi[b], V * sizeof(Shift)));
            TRY(dalloc(ctx, &lv.d2[b], V * sizeof(float)));
            TRY(dalloc(ctx, &lv.chg[b], V));
            CK(cudaMemsetAsync(lv.phi[b], 0, V * sizeof(Shift), ctx->stream));
            launch_fill_f32(lv.d2[b], INFINITY, (long long)V, ctx->stream);
            CK_LAUNCH();
        }
        w = (w + 1) / 2;
        h = (h + 1) / 2;
        if (ctx->cfg.time_subsample)
            tl = (tl + 1) / 2;
    }
    // evaluation / launch / time counters accumulate over the context's life;
    // the per-run counters restart with every upload
    ctx->onion_layers = 0;
    ctx->iter_log.clear();
    std::memset(ctx->outer, 0, sizeof(ctx->outer));
    ctx->uploaded = true;
    ctx->err.clear();
    return VI_OK;
}

vi_status vi_upload(vi_ctx *ctx, const float *rgb, const uint8_t *mask, int W, int H, int T,
                    int ptr_is_device)
{
    // host allocations proportional to the clip may throw; no exception crosses the C ABI
    try {
        return vi_upload_body(ctx, rgb, mask, W, H, T, ptr_is_device);
    } catch (...) {
        return VI_ERR_OOM;
    }
}

vi_status vi_build_pyramid(vi_ctx *ctx)
{
    const Phase ph("pyramid");
    if (!ctx)
        return VI_ERR_ARG;
    if (!ctx->uploaded)
        return fail(ctx, VI_ERR_STATE, "vi_build_pyramid: no upload");
    cudaStream_t st = ctx->stream;
    const int W = ctx->W, H = ctx->H, T = ctx->T;
    const size_t V0 = (size_t)ctx->V0;
    const float s = (float)std::sqrt((double)ctx->cfg.lambda);

    if (ctx->c5) {
        float2 *g = nullptr, *sum = nullptr;
        uint16_t *cnt = nullptr;
        if (!ctx->T0)
            TRY(dalloc(ctx, &ctx->T0, V0 * sizeof(float2)));
        TRY(dalloc(ctx, &g, V0 * sizeof(float2)));
        vi_status r = dalloc(ctx, &sum, V0 * sizeof(float2));
        if (r == VI_OK)
            r = dalloc(ctx, &cnt, V0 * 2 * sizeof(uint16_t));
        if (r == VI_OK) {
            // ctx->tmpA holds the validity bits of the derivative samples
            launch_gradients(ctx->rgb, ctx->mask, W, H, T, g, ctx->tmpA, st);
            launch_box_mean(g, ctx->tmpA, W, H, T, 1 << (ctx->L - 1), sum, cnt, ctx->T0, st);
            cudaStreamSynchronize(st);
        }
        dfree(ctx, g);
        dfree(ctx, sum);
        dfree(ctx, cnt);
        TRY(r);
        CK_LAUNCH();
    }
    launch_level0_channels(ctx->rgb, ctx->mask, ctx->T0, s, ctx->c5, ctx->lv[0].view(), st);
    CK_LAUNCH();
    launch_codes(ctx->lv[0].view(), ctx->tmpA, ctx->tmpB, st);
    CK_LAUNCH();
    for (int l = 1; l < ctx->L; ++l) {
        launch_downsample(ctx->lv[l - 1].view(), ctx->lv[l].view(), l, ctx->T0, W, H, s, ctx->c5,
                          ctx->cfg.time_subsample != 0, st);
        CK_LAUNCH();
        launch_codes(ctx->lv[l].view(), ctx->tmpA, ctx->tmpB, st);
        CK_LAUNCH();
    }
    // FP16 storage: the copies of the screened levels and their magnitude bounds
    for (int l = 0; l < ctx->L; ++l) {
        if (!ctx->lv[l].h4)
            continue;
        CK(cudaMemsetAsync(ctx->lv[l].hmax, 0, 8 * sizeof(unsigned), st));
        launch_shadow_all(ctx->lv[l].view(), st);
        CK_LAUNCH();
    }
    // list sizes of every level (one synchronisation), then the lists
    const uchar3 sets = make_uchar3(CODE_TARGET, CODE_HOLE, CODE_SOURCE);
    std::vector<size_t> base((size_t)ctx->L, 0);
    for (int l = 0; l < ctx->L; ++l) {
        Level &lv = ctx->lv[l];
        if (l > 0)
            base[(size_t)l] = base[(size_t)l - 1] + 3 * (size_t)(compact_blocks(ctx->lv[l - 1].V) + 1);
        launch_compact3_count(lv.code, sets, lv.V, ctx->block_counts + base[(size_t)l], ctx->count_dev + 3 * l, st);
        CK_LAUNCH();
    }
    CK(cudaMemcpyAsync(ctx->host_counts, ctx->count_dev, sizeof(int) * 3 * ctx->L, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int max_list = 1, max_t = 1;
    for (int l = 0; l < ctx->L; ++l) {
        Level &lv = ctx->lv[l];
        dfree(ctx, lv.targets);
        dfree(ctx, lv.holes);
        dfree(ctx, lv.sources);
        lv.nT = ctx->host_counts[3 * l];
        lv.nH = ctx->host_counts[3 * l + 1];
        lv.nS = ctx->host_counts[3 * l + 2];
        if (lv.nS == 0 && lv.nH > 0)
            return fail(ctx, VI_ERR_NO_SOURCE,
                        "no whole known 5x5x5 patch (D~ empty) at level " + std::to_string(l));
        TRY(dalloc(ctx, &lv.targets, sizeof(int) * (size_t)std::max(lv.nT, 1)));
        TRY(dalloc(ctx, &lv.holes, sizeof(int) * (size_t)std::max(lv.nH, 1)));
        TRY(dalloc(ctx, &lv.sources, sizeof(int) * (size_t)std::max(lv.nS, 1)));
        launch_compact3_write(lv.code, sets, lv.V, ctx->block_counts + base[(size_t)l], lv.targets, lv.holes,
                              lv.sources, st);
        CK_LAUNCH();
        max_list = std::max(max_list, lv.nH);
        max_t = std::max(max_t, lv.nT);
    }
    TRY(ensure_partials(ctx, max_list));
    TRY(ensure_partials2(ctx, energy_blocks(max_t)));
    ctx->built = true;
    ctx->hp_ready = false;
    return VI_OK;
}

vi_status vi_init_nnf(vi_ctx *ctx, int level)
{
    if (!ctx)
        return VI_ERR_ARG;
    if (!level_ok(ctx, level))
        return fail(ctx, VI_ERR_ARG, "vi_init_nnf: bad level or no pyramid");
    Level &l = ctx->lv[level];
    if (l.nS == 0)
        return l.nT ? fail(ctx, VI_ERR_NO_SOURCE, "vi_init_nnf: D~ empty") : VI_OK;
    launch_init_nnf(l.view(), l.targets, l.nT, l.sources, l.nS, l.phi[0],
                    (uint32_t)(ctx->cfg.seed & 0xFFFFFFFFull), (uint32_t)(ctx->cfg.seed >> 32),
                    make_tag(PURPOSE_INIT, level, 0), ctx->cfg.clip, ctx->stream);
    CK_LAUNCH();
    return VI_OK;
}

// The onion-peel buffers of the coarsest level (once per context).
static vi_status onion_buffers(vi_ctx *ctx)
{
    Level &l = ctx->lv[ctx->L - 1];
    const size_t V = (size_t)l.V;
    if (!ctx->hp) {
        TRY(dalloc(ctx, &ctx->hp, V));
        TRY(dalloc(ctx, &ctx->layer, V));
        TRY(dalloc(ctx, &ctx->ltgt, V));
        TRY(dalloc(ctx, &ctx->layer_list, V * sizeof(int)));
        TRY(dalloc(ctx, &ctx->ltgt_list, V * sizeof(int)));
    }
    return ctx_ensure_partials(ctx, l.V);
}

// |H'| (ctx->hp at the coarsest level) into *out: one synchronisation.
static vi_status onion_count(vi_ctx *ctx, int *out)
{
    Level &l = ctx->lv[ctx->L - 1];
    cudaStream_t st = ctx->stream;
    launch_count(ctx->hp, l.V, ctx->count_dev + 60, st);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(ctx->host_counts + 60, ctx->count_dev + 60, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *out = ctx->host_counts[60];
    return VI_OK;
}

// One layer of Algorithm 3 on H' = ctx->hp: dH' (H' minus its 3x3x3 erosion),
// the targets (voxels outside H' whose patch meets dH'), the search of
// Algorithm 1 with the partial distance of Eq. 11 (random draws tagged with
// the layer index), and the vote of Eq. 12, which clears the voxels it fills
// from H'; a layer voxel no target reaches stays in H'.
static vi_status onion_step(vi_ctx *ctx, int n_layer)
{
    const int level = ctx->L - 1;
    Level &l = ctx->lv[level];
    const LevelView v = l.view();
    cudaStream_t st = ctx->stream;
    launch_onion_layer(v, ctx->hp, ctx->layer, st);
    launch_onion_targets(v, ctx->hp, ctx->layer, ctx->ltgt, st);
    launch_compact(ctx->layer, 1, l.V, ctx->block_counts, ctx->layer_list, ctx->count_dev + 61, st);
    launch_compact(ctx->ltgt, 1, l.V, ctx->block_counts, ctx->ltgt_list, ctx->count_dev + 62, st);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(ctx->host_counts + 61, ctx->count_dev + 61, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int n_lay = ctx->host_counts[61], n_tgt = ctx->host_counts[62];
    TRY(run_ann(ctx, level, ctx->ltgt_list, n_tgt, ctx->ltgt, 1, ctx->hp, make_tag(PURPOSE_ONION, level, n_layer)));
    VoteArgs a;
    a.L = v;
    a.list = ctx->layer_list;
    a.n = n_lay;
    a.phi = l.phi[0];
    a.d2 = l.d2[0];
    a.allowed = ctx->ltgt;
    a.abit = 1;
    a.weighted = ctx->cfg.weighted;
    a.hp = ctx->hp;
    a.partials = ctx->partials;
    launch_vote(a, ctx->c5, st);
    CK_LAUNCH();
    return VI_OK;
}

vi_status vi_onion_peel(vi_ctx *ctx)
{
    const Phase ph("onion peel");
    if (!ctx)
        return VI_ERR_ARG;
    if (!ctx->built)
        return fail(ctx, VI_ERR_STATE, "vi_onion_peel: no pyramid");
    Level &l = ctx->lv[ctx->L - 1];
    TRY(onion_buffers(ctx));
    launch_extract_bit(l.code, CODE_HOLE, ctx->hp, l.V, ctx->stream);
    CK_LAUNCH();
    int remaining = 0;
    TRY(onion_count(ctx, &remaining));
    int n_layer = 0;
    while (remaining > 0) {
        TRY(onion_step(ctx, n_layer));
        int now = 0;
        TRY(onion_count(ctx, &now));
        ++n_layer;
        if (now >= remaining)
            return fail(ctx, VI_ERR_STATE, "vi_onion_peel: a layer filled no voxel");
        remaining = now;
    }
    ctx->onion_layers = n_layer;
    ctx->hp_ready = false;
    return VI_OK;
}

vi_status vi_onion_layer(vi_ctx *ctx, int layer, const uint8_t *hprime_in, uint8_t *hprime_out, int *n_left)
{
    const Phase ph("onion layer %d", layer);
    if (!ctx)
        return VI_ERR_ARG;
    if (!ctx->built)
        return fail(ctx, VI_ERR_STATE, "vi_onion_layer: no pyramid");
    if (layer < 0 || layer > 0xFFFF)
        return fail(ctx, VI_ERR_ARG, "vi_onion_layer: layer outside [0, 65535]");
    Level &l = ctx->lv[ctx->L - 1];
    TRY(onion_buffers(ctx));
    if (hprime_in) {
        CK(cudaMemcpyAsync(ctx->hp, hprime_in, (size_t)l.V, cudaMemcpyHostToDevice, ctx->stream));
    } else if (!ctx->hp_ready) {
        launch_extract_bit(l.code, CODE_HOLE, ctx->hp, l.V, ctx->stream);
        CK_LAUNCH();
    }
    ctx->hp_ready = true;
    TRY(onion_step(ctx, layer));
    if (hprime_out)
        CK(cudaMemcpyAsync(hprime_out, ctx->hp, (size_t)l.V, cudaMemcpyDeviceToHost, ctx->stream));
    int left = 0;
    TRY(onion_count(ctx, &left));
    if (n_left)
        *n_left = left;
    return VI_OK;
}

vi_status vi_prepare(vi_ctx *ctx)
{
    TRY(vi_build_pyramid(ctx));
    TRY(vi_init_nnf(ctx, ctx->L - 1));
    return vi_onion_peel(ctx);
}

vi_status vi_rescore(vi_ctx *ctx, int level)
{
    if (!ctx)
        return VI_ERR_ARG;
    if (!level_ok(ctx, level))
        return fail(ctx, VI_ERR_ARG, "vi_rescore: bad level or no pyramid");
    Level &l = ctx->lv[level];
    launch_rescore(l.view(), l.targets, l.nT, l.phi[0], l.d2[0], nullptr, ctx->c5, ctx->evals_dev,
                   ctx->stream, rescore_lanes(ctx->cfg.lanes_per_target));
    CK_LAUNCH();
    return VI_OK;
}

vi_status vi_ann(vi_ctx *ctx, int level, int call)
{
    if (!ctx)
        return VI_ERR_ARG;
    if (!level_ok(ctx, level) || call < 0 || call > 0xFFFF)
        return fail(ctx, VI_ERR_ARG, "vi_ann: bad level or call index");
    Level &l = ctx->lv[level];
    return run_ann(ctx, level, l.targets, l.nT, l.code, CODE_TARGET, nullptr,
                   make_tag(PURPOSE_SEARCH, level, call));
}

vi_status vi_reconstruct(vi_ctx *ctx, int level, float *e_host)
{
    if (!ctx)
        return VI_ERR_ARG;
    if (!level_ok(ctx, level))
        return fail(ctx, VI_ERR_ARG, "vi_reconstruct: bad level or no pyramid");
    TRY(vote_level(ctx, level, e_host ? ctx->scal : nullptr));
    if (e_host) {
        CK(cudaMemcpyAsync(ctx->host_scal, ctx->scal, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(ctx->host_evals, ctx->evals_dev, sizeof(ctx->host_evals), cudaMemcpyDeviceToHost,
                           ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        const int nH = ctx->lv[level].nH;
        *e_host = nH ? (float)(ctx->host_scal[0] / (3.0 * nH)) : 0.0f;
    }
    return VI_OK;
}

vi_status vi_iterate(vi_ctx *ctx, int level, int n_outer, int first_call, int *n_done_host,
                     float *e_last_host)
{
    if (!ctx)
        return VI_ERR_ARG;
    if (!level_ok(ctx, level) || first_call < 0)
        return fail(ctx, VI_ERR_ARG, "vi_iterate: bad level or no pyramid");
    const Phase ph("level %d", level);
    int k = 0;
    float e = INFINITY;
    const bool rule = n_outer < 0;
    // with the rule, the cap counts the iterations from call 0, so a run
    // resumed at call first_call stops where the uninterrupted run would
    while (rule ? (e > ctx->cfg.stop && first_call + k < ctx->cfg.max_outer) : (k < n_outer)) {
        const Phase it("L%d iteration %d", level, first_call + k);
        TRY(vi_ann(ctx, level, first_call + k));
        const bool want_e = rule || e_last_host;
        TRY(vi_reconstruct(ctx, level, want_e ? &e : nullptr));
        if (want_e) {
            try {
                ctx->iter_log.push_back({level, first_call + k, e, ctx->host_evals[0] + ctx->host_evals[1]});
            } catch (...) {   // the log is a convenience: a full host heap only shortens it
            }
        }
        ++k;
    }
    if (level < 16)
        ctx->outer[level] += k;
    if (n_done_host)
        *n_done_host = k;
    if (e_last_host)
        *e_last_host = e;
    return VI_OK;
}

vi_status vi_next_level(vi_ctx *ctx, int level)
{
    const Phase ph("transition L%d to L%d", level, level - 1);
    if (!ctx)
        return VI_ERR_ARG;
    if (!level_ok(ctx, level) || level == 0)
        return fail(ctx, VI_ERR_ARG, "vi_next_level: level must be in [1, L)");
    Level &c = ctx->lv[level];
    Level &f = ctx->lv[level - 1];
    launch_upsample_nnf(c.view(), c.phi[0], f.view(), ctx->cfg.time_subsample != 0, f.targets, f.nT, f.sources,
                        f.nS, f.phi[0],
                        (uint32_t)(ctx->cfg.seed & 0xFFFFFFFFull), (uint32_t)(ctx->cfg.seed >> 32),
                        make_tag(PURPOSE_UPSAMPLE, level - 1, 0), ctx->cfg.clip, ctx->stream);
    CK_LAUNCH();
    launch_provisional_fill(c.view(), f.view(), f.holes, f.nH, ctx->c5, ctx->cfg.time_subsample != 0, ctx->stream);
    CK_LAUNCH();
    TRY(vi_rescore(ctx, level - 1));
    return vote_level(ctx, level - 1, nullptr);
}

vi_status vi_final(vi_ctx *ctx)
{
    const Phase ph("final (Eq. 6)");
    if (!ctx)
        return VI_ERR_ARG;
    if (!level_ok(ctx, 0))
        return fail(ctx, VI_ERR_STATE, "vi_final: no pyramid");
    Level &l = ctx->lv[0];
    launch_final(l.view(), l.holes, l.nH, l.phi[0], l.d2[0], ctx->c5, ctx->stream);
    CK_LAUNCH();
    return VI_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint and resume. Between two iterations of Algorithm 4's inner loop
// the state a level carries forward is its channels (u and the texture
// features, known voxels from the pyramid and the occluded ones as last
// voted), its shift map and its distances; every random draw depends only on
// (level, call, voxel), so a run resumed from a saved state draws the same.
// Layout: a header of 16 int32 (magic, version, level, W, H, T, C, then 0),
// then the level's x4 (V float4), x1 (V float, with texture channels), shift
// map (V x 3 int32: dx, dy, dt) and distances (V float).
// ---------------------------------------------------------------------------
namespace {

constexpr int32_t STATE_MAGIC = 0x4B434956;   // "VICK"

size_t state_bytes(vi_ctx *ctx, int level)
{
    const size_t V = (size_t)ctx->lv[level].V;
    return 16 * sizeof(int32_t) + V * (sizeof(float4) + (ctx->c5 ? sizeof(float) : 0) + 3 * sizeof(int32_t) +
                                       sizeof(float));
}

}  // namespace

int vi_iteration_log(vi_ctx *ctx, int cap, int *level, int *call, float *e, unsigned long long *evals)
{
    if (!ctx)
        return -1;
    const int n = (int)ctx->iter_log.size();
    for (int i = 0; i < n && i < cap; ++i) {
        const auto &r = ctx->iter_log[(size_t)i];
        if (level)
            level[i] = r.level;
        if (call)
            call[i] = r.call;
        if (e)
            e[i] = r.e;
        if (evals)
            evals[i] = r.evals;
    }
    return n;
}

size_t vi_state_bytes(vi_ctx *ctx, int level)
{
    if (!ctx || !level_ok(ctx, level))
        return 0;
    return state_bytes(ctx, level);
}

static vi_status vi_save_state_body(vi_ctx *ctx, int level, void *buf, size_t cap)
{
    if (!ctx)
        return VI_ERR_ARG;
    if (!level_ok(ctx, level) || !buf || cap < state_bytes(ctx, level))
        return fail(ctx, VI_ERR_ARG, "vi_save_state: bad level, no pyramid or buffer too small");
    Level &l = ctx->lv[level];
    const size_t V = (size_t)l.V;
    int32_t *hdr = static_cast<int32_t *>(buf);
    std::memset(hdr, 0, 16 * sizeof(int32_t));
    hdr[0] = STATE_MAGIC;
    hdr[1] = 1;
    hdr[2] = level;
    hdr[3] = l.W;
    hdr[4] = l.H;
    hdr[5] = l.T;
    hdr[6] = ctx->c5 ? 5 : 4;
    char *p = static_cast<char *>(buf) + 16 * sizeof(int32_t);
    CK(cudaMemcpyAsync(p, l.x4, V * sizeof(float4), cudaMemcpyDeviceToHost, ctx->stream));
    p += V * sizeof(float4);
    if (ctx->c5) {
        CK(cudaMemcpyAsync(p, l.x1, V * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        p += V * sizeof(float);
    }
    std::vector<Shift> ph(V);
    CK(cudaMemcpyAsync(ph.data(), l.phi[0], V * sizeof(Shift), cudaMemcpyDeviceToHost, ctx->stream));
    char *phi_at = p;
    p += V * 3 * sizeof(int32_t);
    CK(cudaMemcpyAsync(p, l.d2[0], V * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    int32_t *phi = reinterpret_cast<int32_t *>(phi_at);
    for (size_t v = 0; v < V; ++v) {
        phi[3 * v] = ph[v].dx;
        phi[3 * v + 1] = ph[v].dy;
        phi[3 * v + 2] = ph[v].dt;
    }
    return VI_OK;
}

vi_status vi_save_state(vi_ctx *ctx, int level, void *buf, size_t cap)
{
    try {
        return vi_save_state_body(ctx, level, buf, cap);
    } catch (...) {
        return VI_ERR_OOM;
    }
}

static vi_status vi_load_state_body(vi_ctx *ctx, int level, const void *buf, size_t size)
{
    if (!ctx)
        return VI_ERR_ARG;
    if (!level_ok(ctx, level) || !buf || size < 16 * sizeof(int32_t))
        return fail(ctx, VI_ERR_ARG, "vi_load_state: bad level, no pyramid or no buffer");
    Level &l = ctx->lv[level];
    const size_t V = (size_t)l.V;
    const int32_t *hdr = static_cast<const int32_t *>(buf);
    if (hdr[0] != STATE_MAGIC || hdr[1] != 1 || hdr[2] != level || hdr[3] != l.W || hdr[4] != l.H ||
        hdr[5] != l.T || hdr[6] != (ctx->c5 ? 5 : 4) || size != state_bytes(ctx, level))
        return fail(ctx, VI_ERR_ARG, "vi_load_state: the state is of another level, clip or configuration");
    const char *p = static_cast<const char *>(buf) + 16 * sizeof(int32_t);
    CK(cudaMemcpyAsync(l.x4, p, V * sizeof(float4), cudaMemcpyHostToDevice, ctx->stream));
    p += V * sizeof(float4);
    if (ctx->c5) {
        CK(cudaMemcpyAsync(l.x1, p, V * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
        p += V * sizeof(float);
    }
    const int32_t *phi = reinterpret_cast<const int32_t *>(p);
    std::vector<Shift> ph(V);
    for (size_t v = 0; v < V; ++v) {
        if (phi[3 * v] < -32768 || phi[3 * v] > 32767 || phi[3 * v + 1] < -32768 || phi[3 * v + 1] > 32767 ||
            phi[3 * v + 2] < -32768 || phi[3 * v + 2] > 32767)
            return fail(ctx, VI_ERR_ARG, "vi_load_state: shift out of range");
        ph[v].dx = (short)phi[3 * v];
        ph[v].dy = (short)phi[3 * v + 1];
        ph[v].dt = (short)phi[3 * v + 2];
    }
    p += V * 3 * sizeof(int32_t);
    CK(cudaMemcpyAsync(l.phi[0], ph.data(), V * sizeof(Shift), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(l.d2[0], p, V * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    if (l.h4) {
        // the FP16 copies and their magnitude bounds follow the loaded channels
        CK(cudaMemsetAsync(l.hmax, 0, 8 * sizeof(unsigned), ctx->stream));
        launch_shadow_all(l.view(), ctx->stream);
        CK_LAUNCH();
    }
    CK(cudaStreamSynchronize(ctx->stream));   // the host copy of the shifts is released on return
    return VI_OK;
}

vi_status vi_load_state(vi_ctx *ctx, int level, const void *buf, size_t size)
{
    try {
        return vi_load_state_body(ctx, level, buf, size);
    } catch (...) {
        return VI_ERR_OOM;
    }
}

vi_status vi_resume(vi_ctx *ctx, int level, int first_call)
{
    if (!ctx)
        return VI_ERR_ARG;
    if (!level_ok(ctx, level) || first_call < 0)
        return fail(ctx, VI_ERR_ARG, "vi_resume: bad level or no pyramid");
    TRY(vi_iterate(ctx, level, -1, first_call, nullptr, nullptr));
    if (level > 0)
        TRY(vi_next_level(ctx, level));
    for (int l = level - 1; l >= 0; --l) {
        TRY(vi_iterate(ctx, l, -1, 0, nullptr, nullptr));
        if (l > 0)
            TRY(vi_next_level(ctx, l));
    }
    return vi_final(ctx);
}

vi_status vi_run(vi_ctx *ctx)
{
    const Phase ph("inpainting");
    if (!ctx)
        return VI_ERR_ARG;
    TRY(vi_prepare(ctx));
    for (int l = ctx->L - 1; l >= 0; --l) {
        TRY(vi_iterate(ctx, l, -1, 0, nullptr, nullptr));
        if (l > 0)
            TRY(vi_next_level(ctx, l));
    }
    return vi_final(ctx);
}

vi_status vi_energy(vi_ctx *ctx, int level, double *E_H_host, double *E_Ht_host)
{
    if (!ctx)
        return VI_ERR_ARG;
    if (!level_ok(ctx, level))
        return fail(ctx, VI_ERR_ARG, "vi_energy: bad level or no pyramid");
    Level &l = ctx->lv[level];
    const int nb = energy_blocks(std::max(l.nT, 1));
    TRY(ensure_partials2(ctx, nb));
    if (l.nT == 0) {
        if (E_H_host) *E_H_host = 0.0;
        if (E_Ht_host) *E_Ht_host = 0.0;
        return VI_OK;
    }
    launch_energy(l.view(), l.targets, l.nT, l.phi[0], ctx->c5, ctx->partials2, ctx->stream);
    launch_sum_partials2(ctx->partials2, nb, ctx->scal + 2, ctx->stream);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(ctx->host_scal + 2, ctx->scal + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (E_H_host) *E_H_host = ctx->host_scal[2];
    if (E_Ht_host) *E_Ht_host = ctx->host_scal[3];
    return VI_OK;
}

vi_status vi_level_info(vi_ctx *ctx, int level, int *W, int *H, int *T, int *C, long long *n_hole,
                        long long *n_target, long long *n_source)
{
    if (!ctx)
        return VI_ERR_ARG;
    if (!ctx->uploaded || level < 0 || level >= ctx->L)
        return fail(ctx, VI_ERR_ARG, "vi_level_info: bad level or no upload");
    const Level &l = ctx->lv[level];
    if (W) *W = l.W;
    if (H) *H = l.H;
    if (T) *T = l.T;
    if (C) *C = ctx->c5 ? 5 : 3;
    if (n_hole) *n_hole = ctx->built ? l.nH : -1;
    if (n_target) *n_target = ctx->built ? l.nT : -1;
    if (n_source) *n_source = ctx->built ? l.nS : -1;
    return VI_OK;
}

vi_status vi_get_channels(vi_ctx *ctx, int level, float *out, int ptr_is_device)
{
    if (!ctx || !out)
        return VI_ERR_ARG;
    if (!ctx->uploaded || level < 0 || level >= ctx->L)
        return fail(ctx, VI_ERR_ARG, "vi_get_channels: bad level");
    const Level &l = ctx->lv[level];
    const int C = ctx->c5 ? 5 : 3;
    const size_t bytes = (size_t)l.V * C * sizeof(float);
    if (ptr_is_device) {
        launch_get_channels(l.view(), out, C, ctx->stream);
        CK_LAUNCH();
        return VI_OK;
    }
    float *tmp = nullptr;
    TRY(dalloc(ctx, &tmp, bytes));
    launch_get_channels(l.view(), tmp, C, ctx->stream);
    cudaError_t e = cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, tmp);
    if (e != cudaSuccess)
        return fail(ctx, VI_ERR_CUDA, std::string("vi_get_channels: ") + cudaGetErrorString(e));
    return VI_OK;
}

vi_status vi_set_channels(vi_ctx *ctx, int level, const float *in, int ptr_is_device)
{
    if (!ctx || !in)
        return VI_ERR_ARG;
    if (!ctx->uploaded || level < 0 || level >= ctx->L)
        return fail(ctx, VI_ERR_ARG, "vi_set_channels: bad level");
    const Level &l = ctx->lv[level];
    const int C = ctx->c5 ? 5 : 3;
    const size_t bytes = (size_t)l.V * C * sizeof(float);
    if (ptr_is_device) {
        launch_set_channels(l.view(), in, C, ctx->stream);
        launch_shadow_all(l.view(), ctx->stream);
        CK_LAUNCH();
        return VI_OK;
    }
    float *tmp = nullptr;
    TRY(dalloc(ctx, &tmp, bytes));
    cudaError_t e = cudaMemcpyAsync(tmp, in, bytes, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) {
        launch_set_channels(l.view(), tmp, C, ctx->stream);
        launch_shadow_all(l.view(), ctx->stream);
        e = cudaStreamSynchronize(ctx->stream);
    }
    dfree(ctx, tmp);
    if (e != cudaSuccess)
        return fail(ctx, VI_ERR_CUDA, std::string("vi_set_channels: ") + cudaGetErrorString(e));
    return VI_OK;
}

static vi_status vi_get_nnf_body(vi_ctx *ctx, int level, int32_t *phi_host, float *d2_host)
{
    if (!ctx)
        return VI_ERR_ARG;
    if (!level_ok(ctx, level))
        return fail(ctx, VI_ERR_ARG, "vi_get_nnf: bad level or no pyramid");
    const Level &l = ctx->lv[level];
    const size_t V = (size_t)l.V;
    std::vector<Shift> ph(V);
    std::vector<float> dd(V);
    std::vector<uint8_t> code(V);
    CK(cudaMemcpyAsync(ph.data(), l.phi[0], V * sizeof(Shift), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(dd.data(), l.d2[0], V * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(code.data(), l.code, V, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (size_t v = 0; v < V; ++v) {
        const bool t = (code[v] & CODE_TARGET) != 0;
        if (phi_host) {
            phi_host[3 * v] = t ? ph[v].dx : 0;
            phi_host[3 * v + 1] = t ? ph[v].dy : 0;
            phi_host[3 * v + 2] = t ? ph[v].dt : 0;
        }
        if (d2_host)
            d2_host[v] = t ? dd[v] : INFINITY;
    }
    return VI_OK;
}

vi_status vi_get_nnf(vi_ctx *ctx, int level, int32_t *phi_host, float *d2_host)
{
    // host allocations proportional to the clip may throw; no exception crosses the C ABI
    try {
        return vi_get_nnf_body(ctx, level, phi_host, d2_host);
    } catch (...) {
        return VI_ERR_OOM;
    }
}

static vi_status vi_set_nnf_body(vi_ctx *ctx, int level, const int32_t *phi_host, const float *d2_host)
{
    if (!ctx)
        return VI_ERR_ARG;
    if (!level_ok(ctx, level))
        return fail(ctx, VI_ERR_ARG, "vi_set_nnf: bad level or no pyramid");
    const Level &l = ctx->lv[level];
    const size_t V = (size_t)l.V;
    if (phi_host) {
        std::vector<Shift> ph(V);
        for (size_t v = 0; v < V; ++v) {
            const int32_t a = phi_host[3 * v], b = phi_host[3 * v + 1], c = phi_host[3 * v + 2];
            if (a < -32767 || a > 32767 || b < -32767 || b > 32767 || c < -32767 || c > 32767)
                return fail(ctx, VI_ERR_ARG, "vi_set_nnf: shift out of range");
            ph[v].dx = (short)a;
            ph[v].dy = (short)b;
            ph[v].dt = (short)c;
            ph[v].pad = 0;
        }
        CK(cudaMemcpyAsync(l.phi[0], ph.data(), V * sizeof(Shift), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    if (d2_host) {
        CK(cudaMemcpyAsync(l.d2[0], d2_host, V * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return VI_OK;
}

vi_status vi_set_nnf(vi_ctx *ctx, int level, const int32_t *phi_host, const float *d2_host)
{
    // host allocations proportional to the clip may throw; no exception crosses the C ABI
    try {
        return vi_set_nnf_body(ctx, level, phi_host, d2_host);
    } catch (...) {
        return VI_ERR_OOM;
    }
}

vi_status vi_get_masks(vi_ctx *ctx, int level, uint8_t *code_host)
{
    if (!ctx || !code_host)
        return VI_ERR_ARG;
    if (!level_ok(ctx, level))
        return fail(ctx, VI_ERR_ARG, "vi_get_masks: bad level or no pyramid");
    const Level &l = ctx->lv[level];
    CK(cudaMemcpyAsync(code_host, l.code, (size_t)l.V, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return VI_OK;
}

vi_status vi_patch_dist(vi_ctx *ctx, int level, const int32_t *pairs_host, int n, float *out_host)
{
    if (!ctx || (n > 0 && (!pairs_host || !out_host)) || n < 0)
        return VI_ERR_ARG;
    if (!ctx->uploaded || level < 0 || level >= ctx->L)
        return fail(ctx, VI_ERR_ARG, "vi_patch_dist: bad level");
    if (n == 0)
        return VI_OK;
    int *dp = nullptr;
    float *dout = nullptr;
    TRY(dalloc(ctx, &dp, sizeof(int) * 6 * (size_t)n));
    vi_status r = dalloc(ctx, &dout, sizeof(float) * (size_t)n);
    if (r != VI_OK) {
        dfree(ctx, dp);
        return r;
    }
    cudaError_t e = cudaMemcpyAsync(dp, pairs_host, sizeof(int) * 6 * (size_t)n, cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e == cudaSuccess) {
        launch_patch_dist(ctx->lv[level].view(), dp, n, dout, ctx->c5, ctx->stream);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out_host, dout, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, dp);
    dfree(ctx, dout);
    if (e != cudaSuccess)
        return fail(ctx, VI_ERR_CUDA, std::string("vi_patch_dist: ") + cudaGetErrorString(e));
    return VI_OK;
}

vi_status vi_patch_dist_partial(vi_ctx *ctx, int level, const int32_t *pairs_host, int n,
                                const uint8_t *excl_host, float *out_host)
{
    if (!excl_host)
        return vi_patch_dist(ctx, level, pairs_host, n, out_host);
    if (!ctx || (n > 0 && (!pairs_host || !out_host)) || n < 0)
        return VI_ERR_ARG;
    if (!ctx->uploaded || level < 0 || level >= ctx->L)
        return fail(ctx, VI_ERR_ARG, "vi_patch_dist_partial: bad level");
    if (n == 0)
        return VI_OK;
    const size_t V = (size_t)ctx->lv[level].V;
    int *dp = nullptr;
    float *dout = nullptr;
    uint8_t *dex = nullptr;
    TRY(dalloc(ctx, &dp, sizeof(int) * 6 * (size_t)n));
    vi_status r = dalloc(ctx, &dout, sizeof(float) * (size_t)n);
    if (r == VI_OK)
        r = dalloc(ctx, &dex, V);
    if (r != VI_OK) {
        dfree(ctx, dp);
        dfree(ctx, dout);
        return r;
    }
    cudaError_t e = cudaMemcpyAsync(dp, pairs_host, sizeof(int) * 6 * (size_t)n, cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dex, excl_host, V, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) {
        launch_patch_dist_partial(ctx->lv[level].view(), dp, n, dex, dout, ctx->c5, ctx->stream);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out_host, dout, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, dp);
    dfree(ctx, dout);
    dfree(ctx, dex);
    if (e != cudaSuccess)
        return fail(ctx, VI_ERR_CUDA, std::string("vi_patch_dist_partial: ") + cudaGetErrorString(e));
    return VI_OK;
}

vi_status vi_fetch_result(vi_ctx *ctx, float *rgb_out, int ptr_is_device)
{
    if (!ctx || !rgb_out)
        return VI_ERR_ARG;
    if (!ctx->built)
        return fail(ctx, VI_ERR_STATE, "vi_fetch_result: nothing computed");
    const Level &l = ctx->lv[0];
    const size_t bytes = (size_t)l.V * 3 * sizeof(float);
    if (ptr_is_device) {
        launch_pack_rgb(l.view(), rgb_out, ctx->stream);
        CK_LAUNCH();
        return VI_OK;
    }
    if (void *mapped = mapped_host(rgb_out, bytes)) {
        // registered host memory: packed straight into it
        launch_pack_rgb(l.view(), static_cast<float *>(mapped), ctx->stream);
        CK_LAUNCH();
        CK(cudaStreamSynchronize(ctx->stream));
        return VI_OK;
    }
    if (!ctx->out_rgb)
        TRY(dalloc(ctx, &ctx->out_rgb, bytes));
    launch_pack_rgb(l.view(), ctx->out_rgb, ctx->stream);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(rgb_out, ctx->out_rgb, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return VI_OK;
}

vi_status vi_profile(vi_ctx *ctx, int enable)
{
    if (!ctx)
        return VI_ERR_ARG;
    ctx->profiling = enable != 0;
    return VI_OK;
}

vi_status vi_get_stats(vi_ctx *ctx, vi_stats *out)
{
    if (!ctx || !out)
        return VI_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    unsigned long long ev[6] = {0, 0, 0, 0, 0, 0};
    CK(cudaMemcpyAsync(ev, ctx->evals_dev, sizeof(ev), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (size_t i = 0; i < ctx->events_used; ++i) {
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, ctx->events[i].first, ctx->events[i].second));
        ctx->step_ms += ms;
        ctx->step_timed += (unsigned long long)ctx->event_launches[i];
    }
    ctx->events_used = 0;
    out->evals = ev[0] + ev[1];
    out->step_evals = ev[1];
    out->step_gathered = ev[2];
    out->step_gathered_h = ev[3];
    out->screened = ev[4];
    out->screen_passed = ev[5];
    out->step_launches = ctx->step_launches;
    out->step_ms = ctx->step_ms;
    out->step_timed = ctx->step_timed;
    for (int i = 0; i < 16; ++i)
        out->outer[i] = ctx->outer[i];
    out->onion_layers = ctx->onion_layers;
    out->levels = ctx->L;
    out->launches = g_launch_count.load();
    return VI_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Time slabs. One clip's inpainting split by frames over n contexts, each
// holding the whole clip: context r owns the targets and occluded voxels of
// frames [t0_r, t1_r) at every level but the coarsest (which, with the onion
// peel, every context computes alike). Each context searches and votes only
// what it owns; the reads that cross a slab boundary are served by copies:
//  - after every Jacobi sweep, the shifts and change flags of the frame on
//    each side (propagation in t reads the neighbour at t +- 1);
//  - after a search, the shifts and distances of the two frames on each side
//    (the vote reads the patches q in N_p, up to two frames away);
//  - after every vote or provisional fill, the channels of every slab's
//    occluded voxels to every other context (the random search and the
//    patches read anywhere);
//  - the per-voxel changes of every slab into context 0, which sums e over
//    the whole list in the single-context order.
// So every decision, shift, distance and voxel is the same as vi_run's. All
// contexts share one stream on the current device, which orders the copies;
// a multi-device form would use peer copies and events instead.
// ---------------------------------------------------------------------------
namespace {

thread_local std::string g_slab_err;

struct Slab {
    vi_ctx *ctx = nullptr;
    int dev = 0;                          // device of the context
    cudaEvent_t ev = nullptr;             // with a stream per slab: marks its progress for the others
    int t0 = 0, t1 = 0;                   // frames owned
    std::vector<int> tOff, tN, hOff, hN;  // per level: ranges of the target and occluded-voxel lists
    float4 *buf4 = nullptr;               // channels of occluded voxels, indexed like the level's list
    float *buf1 = nullptr;
};

int slab_of(const std::vector<Slab> &S, int t)
{
    for (size_t r = 0; r + 1 < S.size(); ++r)
        if (t < S[r].t1)
            return (int)r;
    return (int)S.size() - 1;
}

// With a stream per slab (possibly on different devices), every stream waits
// for all work issued so far on every other one; with one shared stream,
// stream order already does it.
vi_status barrier(std::vector<Slab> &S)
{
    if (!S[0].ev)
        return VI_OK;
    for (Slab &r : S) {
        vi_ctx *ctx = r.ctx;
        CK(cudaSetDevice(r.dev));
        CK(cudaEventRecord(r.ev, ctx->stream));
    }
    for (Slab &dst : S) {
        vi_ctx *ctx = dst.ctx;
        CK(cudaSetDevice(dst.dev));
        for (Slab &src : S)
            if (&src != &dst)
                CK(cudaStreamWaitEvent(ctx->stream, src.ev, 0));
    }
    return VI_OK;
}

// Slabs on distinct devices exchange through cudaMemcpyPeerAsync between
// buffers of each device's default memory pool (the contexts allocate stream-
// ordered). Peer access enabled with cudaDeviceEnablePeerAccess does not cover
// pool memory: each pool must grant the other devices access itself. For every
// ordered pair of distinct devices that can reach each other, peer access is
// enabled and the owner's default pool grants the peer read/write access;
// pairs that cannot reach each other keep the driver's staged copy.
vi_status grant_peer_access(const std::vector<Slab> &S)
{
    std::vector<int> devs;
    for (const Slab &r : S)
        if (std::find(devs.begin(), devs.end(), r.dev) == devs.end())
            devs.push_back(r.dev);
    for (int owner : devs) {
        cudaMemPool_t pool = nullptr;
        if (cudaDeviceGetDefaultMemPool(&pool, owner) != cudaSuccess) {
            g_slab_err = "vi_run_slabs: no default memory pool on device " + std::to_string(owner);
            return VI_ERR_CUDA;
        }
        for (int peer : devs) {
            if (peer == owner)
                continue;
            int can = 0;
            if (cudaDeviceCanAccessPeer(&can, peer, owner) != cudaSuccess || !can) {
                cudaGetLastError();
                continue;
            }
            if (cudaSetDevice(peer) != cudaSuccess)
                return VI_ERR_CUDA;
            const cudaError_t e = cudaDeviceEnablePeerAccess(owner, 0);
            if (e != cudaSuccess && e != cudaErrorPeerAccessAlreadyEnabled) {
                g_slab_err = std::string("vi_run_slabs: peer access: ") + cudaGetErrorString(e);
                return VI_ERR_CUDA;
            }
            cudaGetLastError();
            cudaMemAccessDesc desc = {};
            desc.location.type = cudaMemLocationTypeDevice;
            desc.location.id = peer;
            desc.flags = cudaMemAccessFlagsProtReadWrite;
            if (cudaMemPoolSetAccess(pool, &desc, 1) != cudaSuccess) {
                g_slab_err = "vi_run_slabs: pool access for device " + std::to_string(peer);
                return VI_ERR_CUDA;
            }
        }
    }
    return VI_OK;
}

// n bytes at src (slab from's device) to dst (slab to's device), on to's stream.
vi_status copy_between(Slab &to, Slab &from, void *dst, const void *src, size_t n, unsigned long long &bytes)
{
    vi_ctx *ctx = to.ctx;
    if (!n || dst == src || !dst || !src)
        return VI_OK;
    CK(cudaSetDevice(to.dev));
    CK(cudaMemcpyPeerAsync(dst, to.dev, src, from.dev, n, ctx->stream));
    bytes += n;
    return VI_OK;
}

// Frames [ta, tb) of a per-voxel array of one context into another's.
template <typename E>
vi_status copy_frames(Slab &to, Slab &from, E *dst, const E *src, int HW, int ta, int tb, unsigned long long &bytes)
{
    if (tb <= ta)
        return VI_OK;
    return copy_between(to, from, dst + (size_t)ta * HW, src + (size_t)ta * HW, (size_t)(tb - ta) * HW * sizeof(E),
                        bytes);
}

// Every slab receives the frames within w of its range from their owners:
// shift buffer b, change-flag buffer b and distance buffer b as selected.
vi_status exchange_halo(std::vector<Slab> &S, int level, int w, int b, bool phi, bool chg, bool d2,
                        unsigned long long &bytes)
{
    const int T = S[0].ctx->lv[level].T, HW = S[0].ctx->lv[level].W * S[0].ctx->lv[level].H;
    TRY(barrier(S));
    for (Slab &dst : S) {
        for (int t = std::max(dst.t0 - w, 0); t < std::min(dst.t1 + w, T); ++t) {
            if (t >= dst.t0 && t < dst.t1)
                continue;
            Slab &src = S[slab_of(S, t)];
            Level &ld = dst.ctx->lv[level], &ls = src.ctx->lv[level];
            if (phi)
                TRY(copy_frames(dst, src, ld.phi[b], ls.phi[b], HW, t, t + 1, bytes));
            if (chg)
                TRY(copy_frames(dst, src, ld.chg[b], ls.chg[b], HW, t, t + 1, bytes));
            if (d2)
                TRY(copy_frames(dst, src, ld.d2[b], ls.d2[b], HW, t, t + 1, bytes));
        }
    }
    return barrier(S);
}

// The channels of every slab's occluded voxels (the only voxels a vote or a
// provisional fill writes) into every other context (all_dst), or into
// context 0 only: packed by the owner, copied, unpacked by the receiver.
vi_status gather_holes(std::vector<Slab> &S, int level, bool all_dst, unsigned long long &bytes)
{
    for (Slab &src : S) {
        vi_ctx *ctx = src.ctx;
        Level &l = ctx->lv[level];
        const int off = src.hOff[level], n = src.hN[level];
        if (!n)
            continue;
        CK(cudaSetDevice(src.dev));
        launch_pack_voxels(l.view(), l.holes + off, n, src.buf4 + off, src.buf1 + off, false, ctx->stream);
        CK_LAUNCH();
    }
    TRY(barrier(S));
    for (Slab &src : S) {
        const int off = src.hOff[level], n = src.hN[level];
        if (!n)
            continue;
        const bool c5 = src.ctx->lv[level].x1 != nullptr;
        for (Slab &dst : S) {
            if (&dst == &src || (!all_dst && &dst != &S[0]))
                continue;
            vi_ctx *ctx = dst.ctx;
            Level &ld = ctx->lv[level];
            TRY(copy_between(dst, src, dst.buf4 + off, src.buf4 + off, sizeof(float4) * (size_t)n, bytes));
            if (c5)
                TRY(copy_between(dst, src, dst.buf1 + off, src.buf1 + off, sizeof(float) * (size_t)n, bytes));
            CK(cudaSetDevice(dst.dev));
            launch_pack_voxels(ld.view(), ld.holes + off, n, dst.buf4 + off, dst.buf1 + off, true, ctx->stream);
            CK_LAUNCH();
        }
    }
    return barrier(S);
}

// The search of one iteration (call) at a sharded level: rescore, n_pm
// sweeps with the halo exchanged after each, copy-back, halo for the vote.
vi_status slab_ann(std::vector<Slab> &S, int level, int call, unsigned long long &bytes)
{
    const Phase ph("slab search L%d call %d", level, call);
    const uint32_t tag = make_tag(PURPOSE_SEARCH, level, call);
    for (Slab &r : S) {
        vi_ctx *ctx = r.ctx;
        Level &l = ctx->lv[level];
        CK(cudaSetDevice(r.dev));
        launch_rescore(l.view(), l.targets + r.tOff[level], r.tN[level], l.phi[0], l.d2[0], nullptr, ctx->c5,
                       ctx->evals_dev, ctx->stream, rescore_lanes(ctx->cfg.lanes_per_target));
        CK_LAUNCH();
    }
    vi_ctx *c0 = S[0].ctx;
    int s = 0;
    for (int k = 1; k <= c0->cfg.n_pm; ++k)
        for (int j = 0; j < c0->cfg.sub_sweeps; ++j, ++s) {
            for (Slab &r : S) {
                vi_ctx *ctx = r.ctx;
                Level &l = ctx->lv[level];
                CK(cudaSetDevice(r.dev));
                TRY(step_launch(ctx, sweep_args(ctx, level, l.targets + r.tOff[level], r.tN[level], l.code,
                                                CODE_TARGET, nullptr, tag, k, j, s)));
            }
            TRY(exchange_halo(S, level, 1, (s + 1) & 1, true, true, false, bytes));
        }
    if (s & 1)
        for (Slab &r : S) {
            vi_ctx *ctx = r.ctx;
            Level &l = ctx->lv[level];
            CK(cudaSetDevice(r.dev));
            launch_copy_targets(l.targets + r.tOff[level], r.tN[level], l.phi[1], l.d2[1], l.phi[0], l.d2[0],
                                ctx->stream);
            CK_LAUNCH();
        }
    return exchange_halo(S, level, 2, 0, true, false, true, bytes);
}

// Votes of every slab, then e over the whole list on context 0 (returned in
// *e when e is not null), then the channels to every context.
vi_status slab_vote(std::vector<Slab> &S, int level, float *e, unsigned long long &bytes)
{
    const Phase ph("slab vote L%d", level);
    for (Slab &r : S) {
        vi_ctx *ctx = r.ctx;
        CK(cudaSetDevice(r.dev));
        TRY(vote_range(ctx, level, r.hOff[level], r.hN[level]));
    }
    vi_ctx *ctx = S[0].ctx;
    if (e) {
        TRY(barrier(S));
        for (size_t i = 1; i < S.size(); ++i)
            TRY(copy_between(S[0], S[i], ctx->partials + S[i].hOff[level], S[i].ctx->partials + S[i].hOff[level],
                             (size_t)S[i].hN[level] * sizeof(float), bytes));
        CK(cudaSetDevice(S[0].dev));
        TRY(sum_changes(ctx, level, ctx->scal));
    }
    TRY(gather_holes(S, level, true, bytes));
    if (e) {
        CK(cudaSetDevice(S[0].dev));
        CK(cudaMemcpyAsync(ctx->host_scal, ctx->scal, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        const int nH = ctx->lv[level].nH;
        *e = nH ? (float)(ctx->host_scal[0] / (3.0 * nH)) : 0.0f;
    }
    return VI_OK;
}

// Level transition (vi_next_level) into sharded level `level` from level + 1.
vi_status slab_next_level(std::vector<Slab> &S, int level, unsigned long long &bytes)
{
    for (Slab &r : S) {
        vi_ctx *ctx = r.ctx;
        Level &c = ctx->lv[level + 1], &f = ctx->lv[level];
        CK(cudaSetDevice(r.dev));
        launch_upsample_nnf(c.view(), c.phi[0], f.view(), false, f.targets + r.tOff[level], r.tN[level], f.sources,
                            f.nS, f.phi[0], (uint32_t)(ctx->cfg.seed & 0xFFFFFFFFull),
                            (uint32_t)(ctx->cfg.seed >> 32), make_tag(PURPOSE_UPSAMPLE, level, 0), ctx->cfg.clip,
                            ctx->stream);
        CK_LAUNCH();
        launch_provisional_fill(c.view(), f.view(), f.holes + r.hOff[level], r.hN[level], ctx->c5, false,
                                ctx->stream);
        CK_LAUNCH();
    }
    TRY(gather_holes(S, level, true, bytes));
    for (Slab &r : S) {
        vi_ctx *ctx = r.ctx;
        Level &f = ctx->lv[level];
        CK(cudaSetDevice(r.dev));
        launch_rescore(f.view(), f.targets + r.tOff[level], r.tN[level], f.phi[0], f.d2[0], nullptr, ctx->c5,
                       ctx->evals_dev, ctx->stream, rescore_lanes(ctx->cfg.lanes_per_target));
        CK_LAUNCH();
    }
    TRY(exchange_halo(S, level, 2, 0, true, false, true, bytes));
    return slab_vote(S, level, nullptr, bytes);
}

// List ranges of every slab at every level (the lists are raster ordered, so
// a slab's entries are contiguous).
vi_status slab_ranges(std::vector<Slab> &S)
{
    vi_ctx *ctx = S[0].ctx;
    CK(cudaSetDevice(S[0].dev));
    for (Slab &r : S) {
        r.tOff.assign(ctx->L, 0);
        r.tN.assign(ctx->L, 0);
        r.hOff.assign(ctx->L, 0);
        r.hN.assign(ctx->L, 0);
    }
    for (int l = 0; l < ctx->L; ++l) {
        Level &lv = ctx->lv[l];
        const int HW = lv.W * lv.H;
        std::vector<int> tl((size_t)lv.nT), hl((size_t)lv.nH);
        if (lv.nT)
            CK(cudaMemcpyAsync(tl.data(), lv.targets, sizeof(int) * tl.size(), cudaMemcpyDeviceToHost, ctx->stream));
        if (lv.nH)
            CK(cudaMemcpyAsync(hl.data(), lv.holes, sizeof(int) * hl.size(), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        for (Slab &r : S) {
            const auto t_a = std::lower_bound(tl.begin(), tl.end(), r.t0 * HW);
            const auto t_b = std::lower_bound(tl.begin(), tl.end(), r.t1 * HW);
            const auto h_a = std::lower_bound(hl.begin(), hl.end(), r.t0 * HW);
            const auto h_b = std::lower_bound(hl.begin(), hl.end(), r.t1 * HW);
            r.tOff[l] = (int)(t_a - tl.begin());
            r.tN[l] = (int)(t_b - t_a);
            r.hOff[l] = (int)(h_a - hl.begin());
            r.hN[l] = (int)(h_b - h_a);
        }
    }
    return VI_OK;
}

vi_status run_slabs(std::vector<Slab> &S, const float *rgb, const uint8_t *mask, int W, int H, int T,
                    int ptr_is_device, float *rgb_out, vi_stats *stats_out, unsigned long long &bytes)
{
    const int n = (int)S.size();
    for (Slab &r : S) {
        vi_ctx *ctx = r.ctx;
        CK(cudaSetDevice(r.dev));
        TRY(vi_upload(ctx, rgb, mask, W, H, T, ptr_is_device));
        // pyramid, initialisation and onion peel, then the coarsest level's
        // iterations: the same on every context
        TRY(vi_prepare(ctx));
        TRY(vi_iterate(ctx, ctx->L - 1, -1, 0, nullptr, nullptr));
    }
    vi_ctx *ctx = S[0].ctx;
    const int L = ctx->L;
    std::vector<unsigned long long> before((size_t)n, 0);
    for (int i = 1; i < n; ++i) {
        vi_stats st;
        CK(cudaSetDevice(S[i].dev));
        TRY(vi_get_stats(S[i].ctx, &st));
        before[(size_t)i] = st.evals;
    }
    TRY(slab_ranges(S));
    int max_h = 1;
    for (int l = 0; l < L; ++l)
        max_h = std::max(max_h, ctx->lv[l].nH);
    for (Slab &r : S) {
        vi_ctx *rc = r.ctx;
        CK(cudaSetDevice(r.dev));
        TRY(dalloc(rc, &r.buf4, sizeof(float4) * (size_t)max_h));
        TRY(dalloc(rc, &r.buf1, sizeof(float) * (size_t)max_h));
    }
    for (int l = L - 2; l >= 0; --l) {
        TRY(slab_next_level(S, l, bytes));
        int k = 0;
        float e = INFINITY;
        while (e > ctx->cfg.stop && k < ctx->cfg.max_outer) {
            TRY(slab_ann(S, l, k, bytes));
            TRY(slab_vote(S, l, &e, bytes));
            ++k;
        }
        if (l < 16)
            ctx->outer[l] += k;
    }
    if (L == 1) {
        CK(cudaSetDevice(S[0].dev));
        TRY(vi_final(ctx));
    } else {
        for (Slab &r : S) {
            Level &l = r.ctx->lv[0];
            CK(cudaSetDevice(r.dev));
            launch_final(l.view(), l.holes + r.hOff[0], r.hN[0], l.phi[0], l.d2[0], r.ctx->c5, r.ctx->stream);
            CK_LAUNCH();
        }
        TRY(gather_holes(S, 0, false, bytes));
    }
    CK(cudaSetDevice(S[0].dev));
    TRY(vi_fetch_result(ctx, rgb_out, ptr_is_device));
    if (stats_out) {
        TRY(vi_get_stats(ctx, stats_out));
        for (int i = 1; i < n; ++i) {
            vi_stats st;
            CK(cudaSetDevice(S[i].dev));
            TRY(vi_get_stats(S[i].ctx, &st));
            stats_out->evals += st.evals - before[(size_t)i];
        }
    }
    return VI_OK;
}

}  // namespace

extern "C" {

const char *vi_slabs_last_error(void) { return g_slab_err.c_str(); }

vi_status vi_run_slabs(const vi_config *cfg, const float *rgb, const uint8_t *mask, int W, int H, int T,
                       int ptr_is_device, int n_slabs, float *rgb_out, vi_stats *stats_out,
                       unsigned long long *exchanged_bytes, void *cuda_stream, const int *devices)
{
    g_slab_err.clear();
    vi_config c;
    if (cfg)
        c = *cfg;
    else
        vi_config_default(&c);
    if (!rgb || !mask || !rgb_out || n_slabs < 1 || n_slabs > 16 || T < n_slabs || c.storage != 0 ||
        c.time_subsample != 0 || (devices && cuda_stream)) {
        g_slab_err = "vi_run_slabs: bad arguments (1 <= n_slabs <= min(16, T); FP32 storage; no temporal "
                     "subsampling; a stream only without devices)";
        return VI_ERR_ARG;
    }
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        g_slab_err = "vi_run_slabs: no CUDA device";
        return VI_ERR_NO_DEVICE;
    }
    if (devices && ptr_is_device && devices[0] != cur) {
        // context 0 writes the result into rgb_out, which is on this device
        g_slab_err = "vi_run_slabs: with device buffers the first slab must be on the current device";
        return VI_ERR_ARG;
    }
    std::vector<Slab> S;
    vi_status st = VI_OK;
    unsigned long long bytes = 0;
    try {
        S.resize((size_t)n_slabs);
        for (int r = 0; r < n_slabs && st == VI_OK; ++r) {
            Slab &sl = S[(size_t)r];
            sl.t0 = (int)((long long)r * T / n_slabs);
            sl.t1 = (int)((long long)(r + 1) * T / n_slabs);
            sl.dev = devices ? devices[r] : cur;
            if (cudaSetDevice(sl.dev) != cudaSuccess) {
                cudaGetLastError();
                st = VI_ERR_ARG;
                g_slab_err = "vi_run_slabs: bad device " + std::to_string(sl.dev);
                break;
            }
            if (devices) {
                // a stream (and an event) of its own on its device
                st = vi_ctx_create(&c, nullptr, &sl.ctx);
                if (st == VI_OK && cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
                    cudaGetLastError();
                    sl.ev = nullptr;
                    st = VI_ERR_CUDA;
                }
            } else {
                // all contexts share one stream: the caller's, else context 0's own
                st = vi_ctx_create(&c, r ? (void *)S[0].ctx->stream : cuda_stream, &sl.ctx);
            }
        }
        if (st == VI_OK && devices)
            st = grant_peer_access(S);
        if (st == VI_OK)
            st = run_slabs(S, rgb, mask, W, H, T, ptr_is_device, rgb_out, stats_out, bytes);
    } catch (...) {
        st = VI_ERR_OOM;
    }
    if (st != VI_OK && g_slab_err.empty()) {
        for (const Slab &r : S)
            if (r.ctx && !r.ctx->err.empty()) {
                g_slab_err = r.ctx->err;
                break;
            }
    }
    if (exchanged_bytes)
        *exchanged_bytes = bytes;
    // every stream drained before any context's memory goes (another
    // context's stream may still read it)
    for (Slab &r : S)
        if (r.ctx && cudaSetDevice(r.dev) == cudaSuccess)
            cudaStreamSynchronize(r.ctx->stream);
    for (size_t r = S.size(); r-- > 0;) {
        Slab &sl = S[r];
        if (cudaSetDevice(sl.dev) != cudaSuccess)
            continue;
        if (sl.ctx) {
            dfree(sl.ctx, sl.buf4);
            dfree(sl.ctx, sl.buf1);
        }
        vi_ctx_destroy(sl.ctx);   // context 0 (the shared stream's owner) last
        if (sl.ev)
            cudaEventDestroy(sl.ev);
    }
    cudaGetLastError();
    cudaSetDevice(cur);
    return st;
}

}  // extern "C"
