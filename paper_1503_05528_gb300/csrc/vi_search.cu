// vi_search.cu -- the spatio-temporal PatchMatch of Sec. 3.1 (Algorithm 1):
// the FP32-storage step kernels (vi_ann.cuh), the distance rescoring of the
// current shifts, the shift-map initialisation and the level transition of
// Sec. 3.6.
#include "vi_ann.cuh"

namespace vi {

void launch_ann_step(const AnnArgs &a, bool c5, cudaStream_t st)
{
    if (a.nT <= 0)
        return;
    VI_COUNT_LAUNCH();
    if (a.L.h4 && !a.excl)
        launch_ann_step_f16(a, c5, st);
    else
        launch_ann_step_impl<false>(a, c5, st);
}

void launch_ann_step_batch(const BatchClip *clips, const int *tprefix, int n, int total_targets, int k,
                           bool c5, bool f16, unsigned long long *ctr, int lanes, cudaStream_t st)
{
    if (total_targets <= 0 || n <= 0)
        return;
    VI_COUNT_LAUNCH();
    if (f16)
        launch_ann_step_batch_f16(clips, tprefix, n, total_targets, k, c5, ctr, lanes, st);
    else
        launch_ann_step_batch_impl<false>(clips, tprefix, n, total_targets, k, c5, ctr, lanes, st);
}

// Distances of the current shifts (buffer 0) for every target of a batch.
template <bool C5, int G>
__global__ void __launch_bounds__(256) k_rescore_batch(const BatchClip *__restrict__ clips,
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
        const LevelView &L = a.L;
        const int p = a.targets[g - __ldg(prefix + c)];
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
    k_rescore_batch<C5, G><<<persistent_grid((long long)total * G), 256, 0, st>>>(clips, tprefix, n, evals);
}

void launch_rescore_batch(const BatchClip *clips, const int *tprefix, int n, int total_targets, bool c5,
                          unsigned long long *evals, int lanes, cudaStream_t st)
{
    if (total_targets <= 0 || n <= 0)
        return;
    VI_COUNT_LAUNCH();
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

template <bool C5, int G, bool PARTIAL>
__global__ void __launch_bounds__(256) k_rescore(LevelView L, const int *__restrict__ targets, int nT,
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

// Sec. 3.6: phi_fine(x, y, t) = (2 dx, 2 dy, dt) of phi_coarse(x/2, y/2, t);
// a shift that does not land in the fine D~ is redrawn uniformly from D~.
__global__ void k_upsample_nnf(LevelView C, const Shift *__restrict__ phi_c, LevelView F,
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
    const Shift pc = phi_c[pt * C.HW + (py >> 1) * C.W + (px >> 1)];
    int dx = 2 * pc.dx, dy = 2 * pc.dy, dt = pc.dt;
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

void launch_upsample_nnf(LevelView coarse, const Shift *phi_c, LevelView fine, const int *targets_f,
                         int nT, const int *sources_f, int nS, Shift *phi_f, uint32_t key0, uint32_t key1,
                         uint32_t tag, uint32_t clip, cudaStream_t st)
{
    if (nT <= 0)
        return;
    VI_COUNT_LAUNCH();
    k_upsample_nnf<<<blocks_for(nT, 256), 256, 0, st>>>(coarse, phi_c, fine, targets_f, nT, sources_f, nS,
                                                        phi_f, key0, key1, tag, clip);
}

// Occluded voxels of the finer level take their coarse parent's channels.
__global__ void k_provisional_fill(LevelView C, LevelView F, const int *__restrict__ holes, int nH, int c5)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nH)
        return;
    const int p = holes[i];
    int px, py, pt;
    decode(p, F.W, F.HW, px, py, pt);
    const int q = pt * C.HW + (py >> 1) * C.W + (px >> 1);
    const float4 a = C.x4[q];
    F.x4[p] = a;
    if (c5)
        F.x1[p] = C.x1[q];
    if (F.h4)
        shadow_store_raise(F, p, a);
}

void launch_provisional_fill(LevelView coarse, LevelView fine, const int *holes_f, int nH, bool c5,
                             cudaStream_t st)
{
    if (nH <= 0)
        return;
    VI_COUNT_LAUNCH();
    k_provisional_fill<<<blocks_for(nH, 256), 256, 0, st>>>(coarse, fine, holes_f, nH, c5 ? 1 : 0);
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
