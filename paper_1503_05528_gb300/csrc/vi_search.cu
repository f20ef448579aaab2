// vi_search.cu -- the spatio-temporal PatchMatch of Sec. 3.1 (Algorithm 1) as
// a parallel (Jacobi) sweep, its shift-map initialisation and the level
// transition of Sec. 3.6.
//
// One thread per target voxel. Targets are raster ordered, so a warp covers a
// run of neighbouring voxels along x; with the piecewise-constant shift maps
// PatchMatch relies on, their candidate source patches are neighbours too, and
// the 5x5x5 gathers of a warp coalesce into contiguous rows.
#include "vi_launch.h"

namespace vi {

static inline int blocks_for(long long n, int block)
{
    long long g = (n + block - 1) / block;
    return (int)(g < 1 ? 1 : g);
}

// Candidate source for target (px, py, pt) under shift (dx, dy, dt): its
// linear index when inside the video and in D~, else -1.
__device__ __forceinline__ int source_of(const LevelView &L, int px, int py, int pt, int dx, int dy,
                                         int dt)
{
    const int sx = px + dx, sy = py + dy, st = pt + dt;
    if (!inside(L, sx, sy, st))
        return -1;
    const int s = st * L.HW + sy * L.W + sx;
    return (L.code[s] & CODE_SOURCE) ? s : -1;
}

template <bool C5>
__global__ void __launch_bounds__(256) k_ann_step(const AnnArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned evals = 0;
    if (i < a.nT) {
        const LevelView &L = a.L;
        const int p = a.targets[i];
        int px, py, pt;
        decode(p, L.W, L.HW, px, py, pt);
        Shift cur = a.phi_in[p];
        float d = a.d_in[p];
        const int sg = (a.k & 1) ? 1 : -1;   // odd k: +1 neighbours; even k: -1

        // propagation: candidates phi(p + sg e_x), phi(p + sg e_y), phi(p + sg e_t)
#pragma unroll 1
        for (int ax = 0; ax < 3; ++ax) {
            const int rx = px + (ax == 0 ? sg : 0);
            const int ry = py + (ax == 1 ? sg : 0);
            const int rt = pt + (ax == 2 ? sg : 0);
            if (!inside(L, rx, ry, rt))
                continue;
            const int r = rt * L.HW + ry * L.W + rx;
            if (!(a.tmask[r] & a.tbit))
                continue;
            const Shift c = a.phi_in[r];
            const int s = source_of(L, px, py, pt, c.dx, c.dy, c.dt);
            if (s < 0)
                continue;
            const float dd = patch_d2<C5>(L, p, px, py, pt, s, a.excl);
            ++evals;
            if (dd < d) {
                d = dd;
                cur = c;
            }
        }

        // random search (Eq. 3)
        const uint4 w = philox4x32_10(make_uint4((uint32_t)p, a.tag | (uint32_t)a.k, a.clip, 0u),
                                      a.key0, a.key1);
        const int shift = a.rho_log2 * a.k + 24;
        const int cdx = cur.dx + random_offset(w.x, a.rmax, shift);
        const int cdy = cur.dy + random_offset(w.y, a.rmax, shift);
        const int cdt = cur.dt + random_offset(w.z, a.rmax, shift);
        const int s = source_of(L, px, py, pt, cdx, cdy, cdt);
        if (s >= 0) {
            const float dd = patch_d2<C5>(L, p, px, py, pt, s, a.excl);
            ++evals;
            if (dd < d) {
                d = dd;
                cur.dx = (short)cdx;
                cur.dy = (short)cdy;
                cur.dt = (short)cdt;
            }
        }
        a.phi_out[p] = cur;
        a.d_out[p] = d;
    }
    count_evals(a.evals, evals);
}

void launch_ann_step(const AnnArgs &a, bool c5, cudaStream_t st)
{
    if (a.nT <= 0)
        return;
    VI_COUNT_LAUNCH();
    if (c5)
        k_ann_step<true><<<blocks_for(a.nT, 256), 256, 0, st>>>(a);
    else
        k_ann_step<false><<<blocks_for(a.nT, 256), 256, 0, st>>>(a);
}

template <bool C5>
__global__ void __launch_bounds__(256) k_rescore(LevelView L, const int *__restrict__ targets, int nT,
                                                 const Shift *__restrict__ phi, float *__restrict__ d_out,
                                                 const uint8_t *excl, unsigned long long *evals_ctr)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned evals = 0;
    if (i < nT) {
        const int p = targets[i];
        int px, py, pt;
        decode(p, L.W, L.HW, px, py, pt);
        const Shift c = phi[p];
        const int s = source_of(L, px, py, pt, c.dx, c.dy, c.dt);
        float d = __int_as_float(0x7f800000);
        if (s >= 0) {
            d = patch_d2<C5>(L, p, px, py, pt, s, excl);
            ++evals;
        }
        d_out[p] = d;
    }
    count_evals(evals_ctr, evals);
}

void launch_rescore(LevelView L, const int *targets, int nT, const Shift *phi, float *d_out,
                    const uint8_t *excl, bool c5, unsigned long long *evals, cudaStream_t st)
{
    if (nT <= 0)
        return;
    VI_COUNT_LAUNCH();
    if (c5)
        k_rescore<true><<<blocks_for(nT, 256), 256, 0, st>>>(L, targets, nT, phi, d_out, excl, evals);
    else
        k_rescore<false><<<blocks_for(nT, 256), 256, 0, st>>>(L, targets, nT, phi, d_out, excl, evals);
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
    F.x4[p] = C.x4[q];
    if (c5)
        F.x1[p] = C.x1[q];
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
