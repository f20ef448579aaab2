// vi_ctx.h -- the context structure behind the vi_ctx handle of the C ABI,
// shared by the single-clip runtime (vi_api.cu) and the batch runtime
// (vi_batch.cu). Internal to the library.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include <cstdio>

#include <nvtx3/nvToolsExt.h>

#include "vi.h"
#include "vi_launch.h"

namespace vi {

// A named NVTX range for the lifetime of the object (phases of the method in
// a profiler's timeline; a no-op unless a tool is attached). The name is
// formatted like printf.
struct Phase {
    explicit Phase(const char *fmt, int a = 0, int b = 0)
    {
        char name[64];
        std::snprintf(name, sizeof(name), fmt, a, b);
        nvtxRangePushA(name);
    }
    ~Phase() { nvtxRangePop(); }
    Phase(const Phase &) = delete;
    Phase &operator=(const Phase &) = delete;
};

// Philox tag word: purpose (4 bits) | level (4) | call (16) | k (8).
enum : uint32_t { PURPOSE_INIT = 1, PURPOSE_SEARCH = 2, PURPOSE_UPSAMPLE = 3, PURPOSE_ONION = 4 };

inline uint32_t make_tag(uint32_t purpose, int level, int call)
{
    return ((purpose & 0xFu) << 28) | (((uint32_t)level & 0xFu) << 24) | (((uint32_t)call & 0xFFFFu) << 8);
}

// Device buffers of one pyramid level.
struct Level {
    int W = 0, H = 0, T = 0;
    int V = 0;
    float4 *x4 = nullptr;
    float *x1 = nullptr;
    uint8_t *code = nullptr;
    uint2 *h4 = nullptr;              // FP16 storage: copy of x4, |x| bounds
    unsigned *hmax = nullptr;
    Shift *phi[2] = {nullptr, nullptr};
    float *d2[2] = {nullptr, nullptr};
    uint8_t *chg[2] = {nullptr, nullptr};   // change flags of the last two sweeps, ping-pong with phi
    int *targets = nullptr, *holes = nullptr, *sources = nullptr;
    int nT = 0, nH = 0, nS = 0;

    LevelView view() const
    {
        LevelView v;
        v.W = W;
        v.H = H;
        v.T = T;
        v.HW = W * H;
        v.V = V;
        v.x4 = x4;
        v.x1 = x1;
        v.code = code;
        v.h4 = h4;
        v.hmax = hmax;
        return v;
    }
};

}  // namespace vi

struct vi_ctx {
    vi_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    bool c5 = true;
    int rho_log2 = 1;

    int W = 0, H = 0, T = 0;
    int V0 = 0;
    int L = 0;
    float *rgb = nullptr;
    uint8_t *mask = nullptr;
    float *out_rgb = nullptr;      // staging of vi_fetch_result to host memory
    float2 *T0 = nullptr;
    std::vector<vi::Level> lv;

    uint8_t *tmpA = nullptr, *tmpB = nullptr;
    int *block_counts = nullptr;
    int *count_dev = nullptr;      // 64 ints
    float *partials = nullptr;     // per-voxel (vote) or per-block reduction scratch
    int partials_cap = 0;
    double *partials2 = nullptr;
    int partials2_cap = 0;
    double *chunks = nullptr;      // chunk sums of the change array (sum_chunks of the largest hole list)
    int chunks_cap = 0;
    double *scal = nullptr;        // device scalars
    double host_scal[8] = {0};     // host copies of scal (read after a stream synchronisation)
    int host_counts[64] = {0};     // host copies of count_dev
    unsigned long long host_evals[6] = {0};   // host copy of evals_dev, read with e
    struct IterRecord {
        int level, call;
        float e;
        unsigned long long evals;   // evaluations of the context so far
    };
    std::vector<IterRecord> iter_log;   // one record per iteration that computed e (since the upload)
    size_t held = 0;                    // device bytes held (checked against cfg.mem_limit)
    std::unordered_map<const void *, size_t> sizes;   // bytes of each allocation
    // [0] rescore evals, [1] step evals, [2] FP32 voxels gathered by the step,
    // [3] FP16 voxels gathered, [4] candidates screened, [5] screened and passed
    unsigned long long *evals_dev = nullptr;

    uint8_t *hp = nullptr, *layer = nullptr, *ltgt = nullptr;   // onion peel: H', dH', its targets
    bool hp_ready = false;         // hp holds the H' left by the last vi_onion_layer
    int *layer_list = nullptr, *ltgt_list = nullptr;

    bool uploaded = false, built = false;
    unsigned long long step_launches = 0;
    int outer[16] = {0};
    int onion_layers = 0;

    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
    std::vector<int> event_launches;   // step launches inside each used event pair
    size_t events_used = 0;
    double step_ms = 0.0;
    unsigned long long step_timed = 0;
};

namespace vi {
// Records a failure on a context (or nothing for a null context).
vi_status ctx_fail(vi_ctx *ctx, vi_status st, const std::string &msg);
// Grows ctx->partials to hold at least n floats.
vi_status ctx_ensure_partials(vi_ctx *ctx, int n);
// Whether the search screens candidates on the FP16 copies at this level:
// always with storage 2; with storage 1 when the level's FP32 channels are
// larger than the L2 cache (smaller levels are served by L2, where halving a
// gather's bytes does not pay for the extra screening gather); never with
// FP32 storage.
bool screen_level(const vi_ctx *ctx, const Level &l);
// Moves a context onto stream st (which the caller keeps owning): its own
// stream, if it had one, is drained and destroyed. Everything the context
// queued before is complete when this returns.
vi_status ctx_adopt_stream(vi_ctx *ctx, cudaStream_t st);
}  // namespace vi
