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

__device__ __forceinline__ unsigned long long shift_key(int dx, int dy, int dt)
{
    return ((unsigned long long)(unsigned short)dx) | ((unsigned long long)(unsigned short)dy << 16) |
           ((unsigned long long)(unsigned short)dt << 32);
}

// Shifts rejected so far in one iteration (at most 3 need remembering).
struct Rejected {
    unsigned long long k0 = ~0ull, k1 = ~0ull, k2 = ~0ull;
    __device__ __forceinline__ bool has(unsigned long long k) const { return k == k0 || k == k1 || k == k2; }
    __device__ __forceinline__ void add(unsigned long long k)
    {
        k2 = k1;
        k1 = k0;
        k0 = k;
    }
};

// ---------------------------------------------------------------------------
// Lane groups. A coarse level has too few targets to fill 152 SMs with one
// thread each, and one thread's candidates are a chain of dependent memory
// round trips. So G consecutive lanes (G = 1, 2, 4, 8; chosen from the target
// count) share a target: they make the same decisions on the same data and
// split each distance's five slices between them (group_d2). PARTIAL selects
// the partial distance of Eq. 11 (onion peel).
// ---------------------------------------------------------------------------
template <int G>
__device__ __forceinline__ unsigned group_mask()
{
    return G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
}

// One candidate of Algorithm 1 for target p: counted as an evaluation when it
// lands in D~ (the oracle counts the same). A candidate equal to the current
// best shift, or to one already rejected in this iteration, has that shift's
// distance, which cannot be strictly smaller than the current best, so it is
// resolved without a gather. Otherwise the G lanes of the group gather its
// distance, bounded by the current best; the decision is the same bit for bit
// as with a full evaluation.
template <bool C5, int G, bool PARTIAL>
__device__ __forceinline__ void try_candidate_g(const AnnArgs &a, int p, int px, int py, int pt, int s,
                                                int cdx, int cdy, int cdt, Shift &cur, float &d,
                                                Rejected &rej, unsigned &evals, unsigned &gathered, int sub,
                                                unsigned gmask)
{
    if (s < 0)
        return;
    ++evals;
    const unsigned long long key = shift_key(cdx, cdy, cdt);
    if (key == shift_key(cur.dx, cur.dy, cur.dt) || rej.has(key))
        return;
    const float dd = group_d2<C5, G, PARTIAL>(a.L, p, px, py, pt, s, a.excl, d, sub, gmask, gathered);
    if (dd < d) {
        d = dd;
        cur.dx = (short)cdx;
        cur.dy = (short)cdy;
        cur.dt = (short)cdt;
    } else {
        rej.add(key);
    }
}

// One PatchMatch iteration k for every target: propagation from the three
// neighbours (Algorithm 1; sign by the parity of k), then the random search
// of Eq. 3 around the propagated shift. Reads phi_in / d_in (the state when
// iteration k began), writes phi_out / d_out. The three neighbours' shifts and
// their sources' set codes are loaded together before any distance.
// The step for target i of the clip described by a (iteration k), by the G
// lanes of one group.
template <bool C5, int G, bool PARTIAL>
__device__ __forceinline__ void ann_one(const AnnArgs &a, int i, int k, int sub, unsigned gmask,
                                        unsigned &evals, unsigned &gathered)
{
    {
        const LevelView &L = a.L;
        const int p = a.targets[i];
        int px, py, pt;
        decode(p, L.W, L.HW, px, py, pt);
        Shift cur = a.phi_in[p];
        float d = a.d_in[p];
        const int sg = (k & 1) ? 1 : -1;   // odd k: +1 neighbours; even k: -1

        // propagation candidates phi(p + sg e_x), phi(p + sg e_y), phi(p + sg e_t)
        const bool in0 = inside(L, px + sg, py, pt), in1 = inside(L, px, py + sg, pt),
                   in2 = inside(L, px, py, pt + sg);
        const int r0 = in0 ? p + sg : p, r1 = in1 ? p + sg * L.W : p, r2 = in2 ? p + sg * L.HW : p;
        const bool t0 = in0 && (a.tmask[r0] & a.tbit), t1 = in1 && (a.tmask[r1] & a.tbit),
                   t2 = in2 && (a.tmask[r2] & a.tbit);
        const Shift c0 = a.phi_in[r0], c1 = a.phi_in[r1], c2 = a.phi_in[r2];
        const int s0 = t0 ? source_of(L, px, py, pt, c0.dx, c0.dy, c0.dt) : -1;
        const int s1 = t1 ? source_of(L, px, py, pt, c1.dx, c1.dy, c1.dt) : -1;
        const int s2 = t2 ? source_of(L, px, py, pt, c2.dx, c2.dy, c2.dt) : -1;
        Rejected rej;
        try_candidate_g<C5, G, PARTIAL>(a, p, px, py, pt, s0, c0.dx, c0.dy, c0.dt, cur, d, rej, evals,
                                        gathered, sub, gmask);
        try_candidate_g<C5, G, PARTIAL>(a, p, px, py, pt, s1, c1.dx, c1.dy, c1.dt, cur, d, rej, evals,
                                        gathered, sub, gmask);
        try_candidate_g<C5, G, PARTIAL>(a, p, px, py, pt, s2, c2.dx, c2.dy, c2.dt, cur, d, rej, evals,
                                        gathered, sub, gmask);

        // random search (Eq. 3)
        const uint4 w = philox4x32_10(make_uint4((uint32_t)p, a.tag | (uint32_t)k, a.clip, 0u),
                                      a.key0, a.key1);
        const int shift = a.rho_log2 * k + 24;
        const int cdx = cur.dx + random_offset(w.x, a.rmax, shift);
        const int cdy = cur.dy + random_offset(w.y, a.rmax, shift);
        const int cdt = cur.dt + random_offset(w.z, a.rmax, shift);
        const int s3 = source_of(L, px, py, pt, cdx, cdy, cdt);
        try_candidate_g<C5, G, PARTIAL>(a, p, px, py, pt, s3, cdx, cdy, cdt, cur, d, rej, evals, gathered,
                                        sub, gmask);
        if (sub == 0) {
            a.phi_out[p] = cur;
            a.d_out[p] = d;
        }
    }
}

template <bool C5, int G, bool PARTIAL>
__global__ void __launch_bounds__(256) k_ann_step(const AnnArgs a)
{
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gt / G;
    const int sub = gt & (G - 1);
    const unsigned gmask = group_mask<G>();
    unsigned evals = 0, gathered = 0;
    if (i < a.nT)
        ann_one<C5, G, PARTIAL>(a, i, a.k, sub, gmask, evals, gathered);
    count_evals(a.evals, sub == 0 ? evals : 0u);
    count_evals(a.gathered, gathered);
}

static int pick_group(int nT);

// Batch form: the targets of n clips in one persistent launch. Clip c owns
// the global target indices [prefix[c], prefix[c+1]) and is described by
// descs[c]; every clip runs iteration k. A grid-stride loop over groups keeps
// the grid at the resident size whatever the batch holds.
template <bool C5, int G>
__global__ void __launch_bounds__(256) k_ann_step_batch(const BatchClip *__restrict__ clips,
                                                        const int *__restrict__ prefix, int n, int k,
                                                        unsigned long long *evals_ctr,
                                                        unsigned long long *gathered_ctr)
{
    const int total = __ldg(prefix + n);
    const int sub = (blockIdx.x * blockDim.x + threadIdx.x) & (G - 1);
    const unsigned gmask = group_mask<G>();
    const int stride = gridDim.x * blockDim.x / G;
    unsigned evals = 0, gathered = 0;
    for (int g = (blockIdx.x * blockDim.x + threadIdx.x) / G; g < total; g += stride) {
        const int c = find_segment(prefix, n, g);
        const AnnArgs &a = (k & 1) ? clips[c].odd : clips[c].even;
        ann_one<C5, G, false>(a, g - __ldg(prefix + c), k, sub, gmask, evals, gathered);
    }
    count_evals(evals_ctr, sub == 0 ? evals : 0u);
    count_evals(gathered_ctr, gathered);
}

// Grid of a persistent batch launch: one wave of 256-thread blocks, or fewer
// when the work is smaller.
static int persistent_grid(long long threads)
{
    static int sms = 0;
    if (sms <= 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 152;
    }
    const long long cap = (long long)sms * 8;   // 8 blocks of 256 threads per SM
    const long long need = (threads + 255) / 256;
    return (int)(need < 1 ? 1 : (need < cap ? need : cap));
}

template <bool C5, int G>
static void launch_ann_step_batch_g(const BatchClip *clips, const int *tprefix, int n, int total, int k,
                                    unsigned long long *evals, unsigned long long *gathered, cudaStream_t st)
{
    k_ann_step_batch<C5, G><<<persistent_grid((long long)total * G), 256, 0, st>>>(clips, tprefix, n, k, evals,
                                                                                  gathered);
}

void launch_ann_step_batch(const BatchClip *clips, const int *tprefix, int n, int total_targets, int k,
                           bool c5, unsigned long long *evals, unsigned long long *gathered, int lanes,
                           cudaStream_t st)
{
    if (total_targets <= 0 || n <= 0)
        return;
    VI_COUNT_LAUNCH();
    switch ((lanes > 0 ? lanes : pick_group(total_targets)) * 2 + (c5 ? 1 : 0)) {
    case 2: launch_ann_step_batch_g<false, 1>(clips, tprefix, n, total_targets, k, evals, gathered, st); break;
    case 3: launch_ann_step_batch_g<true, 1>(clips, tprefix, n, total_targets, k, evals, gathered, st); break;
    case 4: launch_ann_step_batch_g<false, 2>(clips, tprefix, n, total_targets, k, evals, gathered, st); break;
    case 5: launch_ann_step_batch_g<true, 2>(clips, tprefix, n, total_targets, k, evals, gathered, st); break;
    case 8: launch_ann_step_batch_g<false, 4>(clips, tprefix, n, total_targets, k, evals, gathered, st); break;
    case 9: launch_ann_step_batch_g<true, 4>(clips, tprefix, n, total_targets, k, evals, gathered, st); break;
    case 16: launch_ann_step_batch_g<false, 8>(clips, tprefix, n, total_targets, k, evals, gathered, st); break;
    default: launch_ann_step_batch_g<true, 8>(clips, tprefix, n, total_targets, k, evals, gathered, st); break;
    }
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

// Lanes per target: the smallest G in {1, 2, 4, 8} that gives the level at
// least 512 threads per SM. Measured on the 320x240x60 workload (one launch,
// microseconds, G = 1 / 2 / 4 / 8): 445k targets 280 / 301 / 447 / 681,
// 126k targets 101 / 108 / 147 / 207, 40k targets 79 / 51 / 60 / 82, 15k
// targets 78 / 46 / 37 / 34: more lanes pay only while the targets alone
// leave the SMs idle. The partial distance (onion peel, coarsest level, few
// targets) always uses G = 8.
static int pick_group(int nT)
{
    static int sms = 0;
    if (sms <= 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 152;
    }
    const long long want = (long long)sms * 512;
    int G = 1;
    while (G < 8 && (long long)nT * G < want)
        G *= 2;
    return G;
}

template <bool C5, int G, bool PARTIAL>
static void launch_ann_step_g(const AnnArgs &a, cudaStream_t st)
{
    k_ann_step<C5, G, PARTIAL><<<blocks_for((long long)a.nT * G, 256), 256, 0, st>>>(a);
}

void launch_ann_step(const AnnArgs &a, bool c5, cudaStream_t st)
{
    if (a.nT <= 0)
        return;
    VI_COUNT_LAUNCH();
    if (a.excl) {
        if (c5)
            launch_ann_step_g<true, 8, true>(a, st);
        else
            launch_ann_step_g<false, 8, true>(a, st);
        return;
    }
    switch ((a.lanes > 0 ? a.lanes : pick_group(a.nT)) * 2 + (c5 ? 1 : 0)) {
    case 2: launch_ann_step_g<false, 1, false>(a, st); break;
    case 3: launch_ann_step_g<true, 1, false>(a, st); break;
    case 4: launch_ann_step_g<false, 2, false>(a, st); break;
    case 5: launch_ann_step_g<true, 2, false>(a, st); break;
    case 8: launch_ann_step_g<false, 4, false>(a, st); break;
    case 9: launch_ann_step_g<true, 4, false>(a, st); break;
    case 16: launch_ann_step_g<false, 8, false>(a, st); break;
    default: launch_ann_step_g<true, 8, false>(a, st); break;
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
