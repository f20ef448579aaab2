// vi_search.cu -- the spatio-temporal PatchMatch of Sec. 3.1 (Algorithm 1):
// the FP32-storage step kernels (vi_ann.cuh), the distance rescoring of the
// current shifts, the shift-map initialisation and the level transition of
// Sec. 3.6.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "vi.h"
#include "vi_ann.cuh"

namespace vi {

// ---------------------------------------------------------------------------
// Autotuning of the lanes per target. G never changes a result (group_d2 adds
// the slice sums in the same order for every G), so the first launch of a
// kernel family for a given target count is run with every G in {1, 2, 4, 8},
// each writing the same outputs, with its counters pointed at a scratch array:
// one untimed round (module loading, caches) and one timed with events. The
// fastest G is kept for that (device, family, C, storage, target-count bucket
// of a quarter octave); the launch that counts then runs with it. The choice
// depends on the GPU's residency and wave quantisation, which pick_group's
// rule only approximates.
// ---------------------------------------------------------------------------
namespace {

enum TuneFamily : uint32_t { TUNE_STEP = 0, TUNE_STEP_BATCH = 1, TUNE_RESCORE = 2, TUNE_RESCORE_BATCH = 3 };

std::mutex g_tune_mu;
std::map<uint64_t, int> g_tuned;
unsigned long long *g_tune_scratch[64] = {nullptr};

uint64_t tune_key(TuneFamily fam, bool c5, bool f16, long long n)
{
    int dev = 0;
    cudaGetDevice(&dev);
    const int bucket = n > 0 ? (int)std::floor(4.0 * std::log2((double)n)) : 0;
    return ((uint64_t)(uint32_t)dev << 40) | ((uint64_t)fam << 32) | ((uint64_t)(c5 ? 1 : 0) << 31) |
           ((uint64_t)(f16 ? 1 : 0) << 30) | (uint64_t)(uint32_t)bucket;
}

// Scratch counters (8) of the current device, allocated once per process.
unsigned long long *tune_scratch()
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64)
        return nullptr;
    if (!g_tune_scratch[dev]) {
        if (cudaMalloc((void **)&g_tune_scratch[dev], 8 * sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            g_tune_scratch[dev] = nullptr;
        }
    }
    return g_tune_scratch[dev];
}

// The tuned G for key, tuning it first when unknown: launch(G, scratch)
// issues one launch with lanes G and counters at scratch. Returns 0 when the
// tuning could not run (the caller then uses pick_group).
template <typename Launch>
int tuned_lanes(uint64_t key, cudaStream_t st, Launch launch, bool with_warp = false)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end())
        return it->second;
    unsigned long long *scratch = tune_scratch();
    if (!scratch)
        return 0;
    // 32: the warp-shared form of the step (k_ann_step_warp, k_ann_step_batch_warp)
    static const int Gs[5] = {1, 2, 4, 8, 32};
    const int nG = with_warp ? 5 : 4;
    cudaEvent_t ev[6];
    for (int i = 0; i <= nG; ++i)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) {
            for (int j = 0; j < i; ++j)
                cudaEventDestroy(ev[j]);
            cudaGetLastError();
            return 0;
        }
    for (int i = 0; i < nG; ++i)
        launch(Gs[i], scratch);
    cudaEventRecord(ev[0], st);
    for (int i = 0; i < nG; ++i) {
        launch(Gs[i], scratch);
        cudaEventRecord(ev[i + 1], st);
    }
    int best = 0;
    if (cudaEventSynchronize(ev[nG]) == cudaSuccess) {
        float best_ms = 0.0f;
        for (int i = 0; i < nG; ++i) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess && (best == 0 || ms < best_ms)) {
                best = Gs[i];
                best_ms = ms;
            }
        }
    }
    for (int i = 0; i <= nG; ++i)
        cudaEventDestroy(ev[i]);
    if (best)
        g_tuned[key] = best;
    return best;
}

// The tuned G for key, or 0 when the table has none.
int known_lanes(uint64_t key)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(key);
    return it == g_tuned.end() ? 0 : it->second;
}

}  // namespace

}  // namespace vi

extern "C" {

int vi_tune_export(char *buf, int cap)
{
    using namespace vi;
    std::string out;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (const auto &kv : g_tuned) {
            const uint64_t k = kv.first;
            char line[96];
            std::snprintf(line, sizeof(line), "%u %u %u %u %d %d\n", (unsigned)(k >> 40),
                          (unsigned)((k >> 32) & 0xFFu), (unsigned)((k >> 31) & 1u), (unsigned)((k >> 30) & 1u),
                          (int)(int32_t)(uint32_t)(k & 0x3FFFFFFFu), kv.second);
            out += line;
        }
    }
    if (buf && cap > 0) {
        const size_t n = std::min(out.size(), (size_t)cap - 1);
        std::memcpy(buf, out.data(), n);
        buf[n] = '\0';
    }
    return (int)out.size() + 1;
}

vi_status vi_tune_import(const char *text)
{
    using namespace vi;
    if (!text)
        return VI_ERR_ARG;
    std::map<uint64_t, int> add;
    const char *p = text;
    while (*p) {
        unsigned dev, fam, c5, f16;
        int bucket, G, used = 0;
        while (*p == '\n' || *p == ' ' || *p == '\r' || *p == '\t')
            ++p;
        if (!*p)
            break;
        if (std::sscanf(p, "%u %u %u %u %d %d%n", &dev, &fam, &c5, &f16, &bucket, &G, &used) != 6 ||
            dev >= 64 || fam > 3 || c5 > 1 || f16 > 1 || bucket < 0 || bucket > 0x3FFFFFFF ||
            !(G == 1 || G == 2 || G == 4 || G == 8 || (G == 32 && (fam == TUNE_STEP || fam == TUNE_STEP_BATCH))))
            return VI_ERR_ARG;
        add[((uint64_t)dev << 40) | ((uint64_t)fam << 32) | ((uint64_t)c5 << 31) | ((uint64_t)f16 << 30) |
            (uint64_t)bucket] = G;
        p += used;
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto &kv : add)
        g_tuned[kv.first] = kv.second;
    return VI_OK;
}

}  // extern "C"

namespace vi {

void launch_ann_step(const AnnArgs &a, bool c5, cudaStream_t st)
{
    if (a.nT <= 0)
        return;
    VI_COUNT_LAUNCH();
    const bool f16 = a.L.h4 && !a.excl;
    auto run = [&](const AnnArgs &b) {
        if (f16)
            launch_ann_step_f16(b, c5, st);
        else
            launch_ann_step_impl<false>(b, c5, st);
    };
    if (a.lanes > 0 || a.excl) {
        run(a);
        return;
    }
    const uint64_t key = tune_key(TUNE_STEP, c5, f16, a.nT);
    AnnArgs b = a;
    if (a.chg_span == 0) {
        // The first sweeps of a search skip no stale neighbour, so every
        // candidate needs a distance; the later ones skip most. Timing the
        // lane choices on an early sweep favours the forms that do well
        // without the skips, so the table is filled from the first sweep with
        // the change-flag rule on; the sweeps before it use the table when it
        // knows the bucket, else the size rule.
        b.lanes = known_lanes(key);
        run(b);
        return;
    }
    b.lanes = tuned_lanes(key, st, [&](int G, unsigned long long *scr) {
        AnnArgs t = a;
        t.lanes = G;
        t.evals = scr;
        t.gathered = scr + 1;
        t.screen = scr + 2;
        VI_COUNT_LAUNCH();
        run(t);
    }, true);
    run(b);
}

void launch_ann_step_batch(const BatchClip *clips, const int *tprefix, int n, int total_targets, BatchSweep k,
                           bool c5, bool f16, unsigned long long *ctr, int lanes, cudaStream_t st)
{
    if (total_targets <= 0 || n <= 0)
        return;
    VI_COUNT_LAUNCH();
    auto run = [&](int G, unsigned long long *c) {
        if (f16)
            launch_ann_step_batch_f16(clips, tprefix, n, total_targets, k, c5, c, G, st);
        else
            launch_ann_step_batch_impl<false>(clips, tprefix, n, total_targets, k, c5, c, G, st);
    };
    if (lanes <= 0) {
        const uint64_t key = tune_key(TUNE_STEP_BATCH, c5, f16, total_targets);
        // as in launch_ann_step: tuned on the first sweep with the change-flag rule (k >= 3)
        lanes = k.k < 3 ? known_lanes(key)
                      : tuned_lanes(
                            key, st,
                            [&](int G, unsigned long long *scr) {
                                VI_COUNT_LAUNCH();
                                run(G, scr);
                            },
                            true);
    }
    run(lanes, ctr);
}

// Distances of the current shifts (buffer 0) for every target of a batch.
template <bool C5, int G>
__global__ void __launch_bounds__(256, step_min_blocks<G, false>()) k_rescore_batch(const BatchClip *__restrict__ clips,
                                                       const int *__restrict__ prefix, int n,
                                                       unsigned long long *evals_ctr)
{
    const int total = __ldg(prefix + n);
    const int sub = (blockIdx.x * blockDim.x + threadIdx.x) & (G - 1);
    const unsigned gmask = group_mask<G>();
    const int stride = gridDim.x * blockDim.x / G;
    unsigned evals = 0, gathered = 0;
    for (int g = (blockIdx.x * blockDim.x + threadIdx.x) / G; g < total; g += stride) {
        const int c = find_segment(prefix, n, g);
        const AnnArgs &a = clips[c].odd;
        const int i = g - __ldg(prefix + c);
        if (i >= a.nT)
            continue;   // a clip's range is padded to whole warps
        const LevelView L = a.L;   // a register copy (the batch kernels read a from global memory)
        const int p = a.targets[i];
        int px, py, pt;
        decode(p, L.W, L.HW, px, py, pt);
        const Shift f = a.phi_in[p];
        const int s = source_of(L, px, py, pt, f.dx, f.dy, f.dt);
        float d = __int_as_float(0x7f800000);
        if (s >= 0) {
            d = group_d2<C5, G, false>(L, p, px, py, pt, s, nullptr, d, sub, gmask, gathered);
            ++evals;
        }
        if (sub == 0)
            clips[c].d0[p] = d;
    }
    count_evals(evals_ctr, sub == 0 ? evals : 0u);
}

template <bool C5, int G>
static void launch_rescore_batch_g(const BatchClip *clips, const int *tprefix, int n, int total,
                                   unsigned long long *evals, cudaStream_t st)
{
    k_rescore_batch<C5, G><<<persistent_grid((long long)total * G, step_min_blocks<G, false>()), 256, 0, st>>>(
        clips, tprefix, n, evals);
}

static void rescore_batch_g(const BatchClip *clips, const int *tprefix, int n, int total_targets, bool c5,
                            unsigned long long *evals, int lanes, cudaStream_t st)
{
    switch ((lanes > 0 ? lanes : pick_group(total_targets)) * 2 + (c5 ? 1 : 0)) {
    case 2: launch_rescore_batch_g<false, 1>(clips, tprefix, n, total_targets, evals, st); break;
    case 3: launch_rescore_batch_g<true, 1>(clips, tprefix, n, total_targets, evals, st); break;
    case 4: launch_rescore_batch_g<false, 2>(clips, tprefix, n, total_targets, evals, st); break;
    case 5: launch_rescore_batch_g<true, 2>(clips, tprefix, n, total_targets, evals, st); break;
    case 8: launch_rescore_batch_g<false, 4>(clips, tprefix, n, total_targets, evals, st); break;
    case 9: launch_rescore_batch_g<true, 4>(clips, tprefix, n, total_targets, evals, st); break;
    case 16: launch_rescore_batch_g<false, 8>(clips, tprefix, n, total_targets, evals, st); break;
    default: launch_rescore_batch_g<true, 8>(clips, tprefix, n, total_targets, evals, st); break;
    }
}

void launch_rescore_batch(const BatchClip *clips, const int *tprefix, int n, int total_targets, bool c5,
                          unsigned long long *evals, int lanes, cudaStream_t st)
{
    if (total_targets <= 0 || n <= 0)
        return;
    VI_COUNT_LAUNCH();
    if (lanes <= 0)
        lanes = tuned_lanes(tune_key(TUNE_RESCORE_BATCH, c5, false, total_targets), st,
                            [&](int G, unsigned long long *scr) {
                                VI_COUNT_LAUNCH();
                                rescore_batch_g(clips, tprefix, n, total_targets, c5, scr, G, st);
                            });
    rescore_batch_g(clips, tprefix, n, total_targets, c5, evals, lanes, st);
}

template <bool C5, int G, bool PARTIAL>
__global__ void __launch_bounds__(256, step_min_blocks<G, PARTIAL>()) k_rescore(LevelView L, const int *__restrict__ targets, int nT,
                                                 const Shift *__restrict__ phi, float *__restrict__ d_out,
                                                 const uint8_t *excl, unsigned long long *evals_ctr)
{
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gt / G;
    const int sub = gt & (G - 1);
    const unsigned gmask = group_mask<G>();
    unsigned evals = 0, gathered = 0;
    if (i < nT) {
        const int p = targets[i];
        int px, py, pt;
        decode(p, L.W, L.HW, px, py, pt);
        const Shift c = phi[p];
        const int s = source_of(L, px, py, pt, c.dx, c.dy, c.dt);
        float d = __int_as_float(0x7f800000);
        if (s >= 0) {
            d = group_d2<C5, G, PARTIAL>(L, p, px, py, pt, s, excl, d, sub, gmask, gathered);
            ++evals;
        }
        if (sub == 0)
            d_out[p] = d;
    }
    count_evals(evals_ctr, sub == 0 ? evals : 0u);
}

template <bool C5, int G, bool PARTIAL>
static void launch_rescore_g(LevelView L, const int *targets, int nT, const Shift *phi, float *d_out,
                             const uint8_t *excl, unsigned long long *evals, cudaStream_t st)
{
    k_rescore<C5, G, PARTIAL><<<blocks_for((long long)nT * G, 256), 256, 0, st>>>(L, targets, nT, phi,
                                                                                  d_out, excl, evals);
}

static void rescore_g(LevelView L, const int *targets, int nT, const Shift *phi, float *d_out, bool c5,
                      unsigned long long *evals, cudaStream_t st, int lanes)
{
    const uint8_t *excl = nullptr;
    switch ((lanes > 0 ? lanes : pick_group(nT)) * 2 + (c5 ? 1 : 0)) {
    case 2: launch_rescore_g<false, 1, false>(L, targets, nT, phi, d_out, excl, evals, st); break;
    case 3: launch_rescore_g<true, 1, false>(L, targets, nT, phi, d_out, excl, evals, st); break;
    case 4: launch_rescore_g<false, 2, false>(L, targets, nT, phi, d_out, excl, evals, st); break;
    case 5: launch_rescore_g<true, 2, false>(L, targets, nT, phi, d_out, excl, evals, st); break;
    case 8: launch_rescore_g<false, 4, false>(L, targets, nT, phi, d_out, excl, evals, st); break;
    case 9: launch_rescore_g<true, 4, false>(L, targets, nT, phi, d_out, excl, evals, st); break;
    case 16: launch_rescore_g<false, 8, false>(L, targets, nT, phi, d_out, excl, evals, st); break;
    default: launch_rescore_g<true, 8, false>(L, targets, nT, phi, d_out, excl, evals, st); break;
    }
}

void launch_rescore(LevelView L, const int *targets, int nT, const Shift *phi, float *d_out,
                    const uint8_t *excl, bool c5, unsigned long long *evals, cudaStream_t st, int lanes)
{
    if (nT <= 0)
        return;
    VI_COUNT_LAUNCH();
    if (excl) {
        if (c5)
            launch_rescore_g<true, 8, true>(L, targets, nT, phi, d_out, excl, evals, st);
        else
            launch_rescore_g<false, 8, true>(L, targets, nT, phi, d_out, excl, evals, st);
        return;
    }
    // k_rescore reads only the shifts and the channels, so every tuning launch
    // writes the same distances
    if (lanes <= 0)
        lanes = tuned_lanes(tune_key(TUNE_RESCORE, c5, false, nT), st, [&](int G, unsigned long long *scr) {
            VI_COUNT_LAUNCH();
            rescore_g(L, targets, nT, phi, d_out, c5, scr, st, G);
        });
    rescore_g(L, targets, nT, phi, d_out, c5, evals, st, lanes);
}

__global__ void k_copy_targets(const int *__restrict__ targets, int nT, const Shift *__restrict__ ps,
                               const float *__restrict__ ds, Shift *__restrict__ pd, float *__restrict__ dd)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nT) {
        const int p = targets[i];
        pd[p] = ps[p];
        dd[p] = ds[p];
    }
}

void launch_copy_targets(const int *targets, int nT, const Shift *phi_src, const float *d_src,
                         Shift *phi_dst, float *d_dst, cudaStream_t st)
{
    if (nT <= 0)
        return;
    VI_COUNT_LAUNCH();
    k_copy_targets<<<blocks_for(nT, 256), 256, 0, st>>>(targets, nT, phi_src, d_src, phi_dst, d_dst);
}

// Shift-map initialisation: a uniform source of D~ for every target (word 0
// of Philox with counter (voxel, tag, clip, 0)).
__global__ void k_init_nnf(LevelView L, const int *__restrict__ targets, int nT,
                           const int *__restrict__ sources, int nS, Shift *__restrict__ phi,
                           uint32_t k0, uint32_t k1, uint32_t tag, uint32_t clip)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nT)
        return;
    const int p = targets[i];
    int px, py, pt, sx, sy, st;
    decode(p, L.W, L.HW, px, py, pt);
    const uint4 w = philox4x32_10(make_uint4((uint32_t)p, tag, clip, 0u), k0, k1);
    const int s = sources[uniform_index(w.x, (uint32_t)nS)];
    decode(s, L.W, L.HW, sx, sy, st);
    Shift c;
    c.dx = (short)(sx - px);
    c.dy = (short)(sy - py);
    c.dt = (short)(st - pt);
    c.pad = 0;
    phi[p] = c;
}

void launch_init_nnf(LevelView L, const int *targets, int nT, const int *sources, int nS, Shift *phi,
                     uint32_t key0, uint32_t key1, uint32_t tag, uint32_t clip, cudaStream_t st)
{
    if (nT <= 0)
        return;
    VI_COUNT_LAUNCH();
    k_init_nnf<<<blocks_for(nT, 256), 256, 0, st>>>(L, targets, nT, sources, nS, phi, key0, key1, tag,
                                                    clip);
}

// Sec. 3.6: phi_fine(x, y, t) = (2 dx, 2 dy, dt) of phi_coarse(x/2, y/2, t)
// (with tsub, the temporal subsampling option: (2 dx, 2 dy, 2 dt) of
// phi_coarse(x/2, y/2, t/2)); a shift that does not land in the fine D~ is
// redrawn uniformly from D~.
__global__ void k_upsample_nnf(LevelView C, const Shift *__restrict__ phi_c, LevelView F, int tsub,
                               const int *__restrict__ targets, int nT, const int *__restrict__ sources,
                               int nS, Shift *__restrict__ phi_f, uint32_t k0, uint32_t k1, uint32_t tag,
                               uint32_t clip)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nT)
        return;
    const int p = targets[i];
    int px, py, pt;
    decode(p, F.W, F.HW, px, py, pt);
    const Shift pc = phi_c[(tsub ? pt >> 1 : pt) * C.HW + (py >> 1) * C.W + (px >> 1)];
    int dx = 2 * pc.dx, dy = 2 * pc.dy, dt = tsub ? 2 * pc.dt : pc.dt;
    if (source_of(F, px, py, pt, dx, dy, dt) < 0) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)p, tag, clip, 0u), k0, k1);
        const int s = sources[uniform_index(w.x, (uint32_t)nS)];
        int sx, sy, st;
        decode(s, F.W, F.HW, sx, sy, st);
        dx = sx - px;
        dy = sy - py;
        dt = st - pt;
    }
    Shift c;
    c.dx = (short)dx;
    c.dy = (short)dy;
    c.dt = (short)dt;
    c.pad = 0;
    phi_f[p] = c;
}

void launch_upsample_nnf(LevelView coarse, const Shift *phi_c, LevelView fine, bool tsub, const int *targets_f,
                         int nT, const int *sources_f, int nS, Shift *phi_f, uint32_t key0, uint32_t key1,
                         uint32_t tag, uint32_t clip, cudaStream_t st)
{
    if (nT <= 0)
        return;
    VI_COUNT_LAUNCH();
    k_upsample_nnf<<<blocks_for(nT, 256), 256, 0, st>>>(coarse, phi_c, fine, tsub ? 1 : 0, targets_f, nT,
                                                        sources_f, nS, phi_f, key0, key1, tag, clip);
}

// Occluded voxels of the finer level take their coarse parent's channels.
__global__ void k_provisional_fill(LevelView C, LevelView F, const int *__restrict__ holes, int nH, int c5,
                                   int tsub)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nH)
        return;
    const int p = holes[i];
    int px, py, pt;
    decode(p, F.W, F.HW, px, py, pt);
    const int q = (tsub ? pt >> 1 : pt) * C.HW + (py >> 1) * C.W + (px >> 1);
    const float4 a = C.x4[q];
    F.x4[p] = a;
    if (c5)
        F.x1[p] = C.x1[q];
    if (F.h4)
        shadow_store_raise(F, p, a);
}

void launch_provisional_fill(LevelView coarse, LevelView fine, const int *holes_f, int nH, bool c5, bool tsub,
                             cudaStream_t st)
{
    if (nH <= 0)
        return;
    VI_COUNT_LAUNCH();
    k_provisional_fill<<<blocks_for(nH, 256), 256, 0, st>>>(coarse, fine, holes_f, nH, c5 ? 1 : 0,
                                                            tsub ? 1 : 0);
}

template <bool C5>
__global__ void k_patch_dist(LevelView L, const int *__restrict__ pairs, int n, float *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const int *q = pairs + 6 * i;
    const int px = q[0], py = q[1], pt = q[2], sx = q[3], sy = q[4], st = q[5];
    float d = __int_as_float(0x7f800000);
    const bool src_ok = sx >= 2 && sx < L.W - 2 && sy >= 2 && sy < L.H - 2 && st >= 2 && st < L.T - 2;
    if (src_ok && inside(L, px, py, pt)) {
        const int p = pt * L.HW + py * L.W + px;
        const int s = st * L.HW + sy * L.W + sx;
        d = patch_d2<C5>(L, p, px, py, pt, s, nullptr);
    }
    out[i] = d;
}

// The partial distance of Eq. 11 for (target, source) pairs, through the
// function the onion peel's search uses (group_d2 with PARTIAL, here by one
// lane): target voxels with excl != 0 are left out, the sum is divided by the
// count kept (+inf when none is).
template <bool C5>
__global__ void k_patch_dist_partial(LevelView L, const int *__restrict__ pairs, int n,
                                     const uint8_t *__restrict__ excl, float *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float d = __int_as_float(0x7f800000);
    if (i < n) {
        const int *q = pairs + 6 * i;
        const int px = q[0], py = q[1], pt = q[2], sx = q[3], sy = q[4], st = q[5];
        const bool src_ok = sx >= 2 && sx < L.W - 2 && sy >= 2 && sy < L.H - 2 && st >= 2 && st < L.T - 2;
        if (src_ok && inside(L, px, py, pt)) {
            const int p = pt * L.HW + py * L.W + px;
            const int s = st * L.HW + sy * L.W + sx;
            unsigned gathered = 0;
            d = group_d2<C5, 1, true>(L, p, px, py, pt, s, excl, __int_as_float(0x7f800000), 0,
                                      1u << (threadIdx.x & 31), gathered);
        }
        out[i] = d;
    }
}

void launch_patch_dist_partial(LevelView L, const int *pairs, int n, const uint8_t *excl, float *out, bool c5,
                               cudaStream_t st)
{
    if (n <= 0)
        return;
    VI_COUNT_LAUNCH();
    if (c5)
        k_patch_dist_partial<true><<<blocks_for(n, 256), 256, 0, st>>>(L, pairs, n, excl, out);
    else
        k_patch_dist_partial<false><<<blocks_for(n, 256), 256, 0, st>>>(L, pairs, n, excl, out);
}

void launch_patch_dist(LevelView L, const int *pairs, int n, float *out, bool c5, cudaStream_t st)
{
    if (n <= 0)
        return;
    VI_COUNT_LAUNCH();
    if (c5)
        k_patch_dist<true><<<blocks_for(n, 256), 256, 0, st>>>(L, pairs, n, out);
    else
        k_patch_dist<false><<<blocks_for(n, 256), 256, 0, st>>>(L, pairs, n, out);
}

}  // namespace vi
