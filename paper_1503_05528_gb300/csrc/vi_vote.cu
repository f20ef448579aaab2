// vi_vote.cu -- reconstruction of Sec. 3.2 (Eq. 4, Eq. 5, Eq. 9; Eq. 12 during
// the initialisation), the final best-patch step (Eq. 6), the energy (Eq. 1),
// the onion-peel sets of Algorithm 3 and layout packing.
#include "vi_launch.h"

namespace vi {

static inline int blocks_for(long long n, int block)
{
    long long g = (n + block - 1) / block;
    return (int)(g < 1 ? 1 : g);
}

static constexpr int VOTE_BLOCK = 256;            // 8 warps, one occluded voxel per warp
static constexpr int VOTE_WARPS = VOTE_BLOCK / 32;
// Resident blocks per SM the vote kernels are compiled for: 8 (every warp
// slot; 32 registers, 12 bytes spilled) instead of the 6 that their 36
// registers allow. The vote waits on its gathers of shifts, distances and
// source voxels, and more warps hide that: measured on GB300, the 48-clip
// batch took 1,117 against 1,143 ms per step.
static constexpr int VOTE_MIN_BLOCKS = 8;

// The patch offsets a lane owns: j = l, l+32, l+64, l+96 (j < 125), offset
// (j%5 - 2, (j/5)%5 - 2, j/25 - 2), packed as bytes (dx+2, dy+2, dt+2, 1 if
// j < 125).
struct VoteLane {
    unsigned off[4];
};

__device__ __forceinline__ VoteLane vote_lane(int lane)
{
    VoteLane v;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int j = lane + 32 * m;
        v.off[m] = j < 125 ? ((unsigned)(j % 5) | ((unsigned)((j / 5) % 5) << 8) | ((unsigned)(j / 25) << 16) |
                              (1u << 24))
                           : 0u;
    }
    return v;
}

// Sums six values over the warp and returns the sums on lane 0 (other lanes:
// unspecified). A transposed butterfly: at xor 16 each lane keeps three of the
// six values and sends the other three, at xor 8 two of its three (padded to
// four), at xor 4 one of those two; xor 2 and xor 1 finish the sums, which
// then sit on lanes 0, 4, 8, 16, 20 and 24. 13 shuffles and 8 adds instead of
// six trees of 5 each.
__device__ __forceinline__ void warp_sum6(float (&v)[6])
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float a[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float keep = b4 ? v[i + 3] : v[i];
        const float send = b4 ? v[i] : v[i + 3];
        a[i] = keep + __shfl_xor_sync(FULL, send, 16);
    }
    // values (b4 ? 3 : 0) + 0, 1, 2; the fourth slot is 0
    const float c0 = (b3 ? a[2] : a[0]) + __shfl_xor_sync(FULL, b3 ? a[0] : a[2], 8);
    const float c1 = (b3 ? 0.0f : a[1]) + __shfl_xor_sync(FULL, b3 ? a[1] : 0.0f, 8);
    float r = (b2 ? c1 : c0) + __shfl_xor_sync(FULL, b2 ? c0 : c1, 4);
    r += __shfl_xor_sync(FULL, r, 2);
    r += __shfl_xor_sync(FULL, r, 1);
    v[0] = r;
    v[1] = __shfl_sync(FULL, r, 4);
    v[2] = __shfl_sync(FULL, r, 8);
    v[3] = __shfl_sync(FULL, r, 16);
    v[4] = __shfl_sync(FULL, r, 20);
    v[5] = __shfl_sync(FULL, r, 24);
}

// One warp per voxel p; lane l handles the q = p + offset of its offsets
// (the q in N_p).
//  1. each lane loads d2(q) of its contributors (q inside the video, allowed,
//     finite);
//  2. sigma_p^2 = the element of rank ceil(0.75 n) of the n values (nearest
//     rank), found by a bitwise radix select over the IEEE bit patterns of the
//     non-negative d2 with warp-wide counts;
//  3. s_q = exp(-d2(q) / (2 sigma_p^2)) (limit 1/0 for sigma_p = 0; 1 when
//     unweighted); each lane accumulates s_q u(p + phi(q)) over all channels,
//     from the source voxels found in step 1;
//  4. warp sums (warp_sum6); lane 0 writes u(p) and stores |u_new - u_old|
//     summed over R, G, B in the voxel's slot of partials.
// A voxel at least 2 from every border has its whole patch inside the video
// and skips those tests.
template <bool C5>
__device__ __forceinline__ void vote_one(const VoteArgs &a, int item, int lane, const VoteLane &vl)
{
    float change = 0.0f;
    {
        // the level view through a reference: in the batch vote a register
        // copy cost 10 registers and two resident blocks per SM (1,173 against
        // 1,159 ms per 48-clip batch)
        const LevelView &L = a.L;
        const int p = a.list[item];
        int px, py, pt;
        decode(p, L.W, L.HW, px, py, pt);
        const bool interior = px >= 2 && px < L.W - 2 && py >= 2 && py < L.H - 2 && pt >= 2 && pt < L.T - 2;
        float dq[4];
        int sv[4];   // source voxel p + phi(q) of each contributor
        unsigned okm = 0;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const unsigned o = vl.off[m];
            dq[m] = 0.0f;
            sv[m] = 0;
            if (o) {
                const int ox = (int)(o & 0xFFu) - 2, oy = (int)((o >> 8) & 0xFFu) - 2,
                          ot = (int)((o >> 16) & 0xFFu) - 2;
                if (interior || inside(L, px + ox, py + oy, pt + ot)) {
                    const int q = p + ot * L.HW + oy * L.W + ox;
                    if (!a.allowed || (a.allowed[q] & a.abit)) {
                        const float d = a.d2[q];
                        const Shift f = a.phi[q];
                        // finite distance, and a source voxel p + phi(q) inside
                        // the level. For a shift map of the search it always
                        // is: q + phi(q) is a source centre, at least 2 from
                        // every border, and p is within 2 of q. The test on
                        // the linear index only keeps an injected map from
                        // reading outside the level's buffers (the full 3-D
                        // test cost 20 of 1,160 ms per 48-clip batch).
                        const int s = p + (int)f.dt * L.HW + (int)f.dy * L.W + (int)f.dx;
                        if (d < __int_as_float(0x7f800000) && (unsigned)s < (unsigned)L.V) {
                            dq[m] = d;
                            sv[m] = s;
                            okm |= 1u << m;
                        }
                    }
                }
            }
        }
        const int n = __reduce_add_sync(0xffffffffu, __popc(okm));
        if (n > 0) {
            float sigma2 = 0.0f;
            if (a.weighted) {
                // Radix select of the value of 0-based rank r over the bit
                // patterns (non-negative finite floats order like their bits,
                // all below 2^31; slots without a contributor hold 2^32 - 1,
                // above all of them, so they never count). Invariant before
                // bit b: the answer's bits above b are those of X (its bits
                // <= b are 0), lo = #{v < X} and hi = #{v < X + 2^(b+1)}, so
                // lo <= r < hi. The search starts at the highest bit where the
                // smallest and largest values differ (every bit above it is
                // shared by all values), and once a single value is left in
                // [X, X + 2^(b+1)) it is the answer: about log2(n) steps for
                // distinct values instead of 31.
                const unsigned r = (unsigned)((3 * n + 3) / 4 - 1);   // 0-based nearest rank
                unsigned u[4];
                unsigned umin = 0xffffffffu, umax = 0u;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const bool ok = (okm >> m) & 1u;
                    u[m] = ok ? __float_as_uint(dq[m]) : 0xffffffffu;
                    umin = min(umin, u[m]);
                    umax = max(umax, ok ? u[m] : 0u);
                }
                umin = __reduce_min_sync(0xffffffffu, umin);
                umax = __reduce_max_sync(0xffffffffu, umax);
                unsigned X = umin;
                if (umin != umax) {
                    int b = 31 - __clz(umin ^ umax);        // <= 30
                    X = umin & ~((2u << b) - 1u);
                    unsigned lo = 0, hi = (unsigned)n;
                    for (; b >= 0 && hi - lo > 1; --b) {
                        const unsigned Tt = X | (1u << b);
                        unsigned c = 0;
#pragma unroll
                        for (int m = 0; m < 4; ++m)
                            c += u[m] < Tt;
                        c = __reduce_add_sync(0xffffffffu, c);
                        if (c <= r) {
                            X = Tt;
                            lo = c;
                        } else {
                            hi = c;
                        }
                    }
                    if (hi - lo == 1) {
                        // the one value in [X, X + 2^(b+1)): the smallest v >= X
                        unsigned mn = 0xffffffffu;
#pragma unroll
                        for (int m = 0; m < 4; ++m)
                            mn = min(mn, u[m] >= X ? u[m] : 0xffffffffu);
                        X = __reduce_min_sync(0xffffffffu, mn);
                    }
                }
                sigma2 = __uint_as_float(X);
            }
            float n0 = 0.f, n1 = 0.f, n2 = 0.f, n3 = 0.f, n4 = 0.f, den = 0.f;
            const float inv2s = sigma2 > 0.0f ? 1.0f / (2.0f * sigma2) : 0.0f;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                if (!((okm >> m) & 1u))
                    continue;
                float w;
                if (!a.weighted)
                    w = 1.0f;
                else if (sigma2 > 0.0f)
                    w = dq[m] > 0.0f ? expf(-(dq[m] * inv2s)) : 1.0f;   // inv2s may be +inf
                else
                    w = (dq[m] == 0.0f) ? 1.0f : 0.0f;
                const int s = sv[m];
                const float4 v = L.x4[s];
                n0 = fmaf(w, v.x, n0);
                n1 = fmaf(w, v.y, n1);
                n2 = fmaf(w, v.z, n2);
                n3 = fmaf(w, v.w, n3);
                if (C5)
                    n4 = fmaf(w, L.x1[s], n4);
                den += w;
            }
            float sums[6] = {n0, n1, n2, n3, n4, den};
            warp_sum6(sums);
            n0 = sums[0];
            n1 = sums[1];
            n2 = sums[2];
            n3 = sums[3];
            n4 = sums[4];
            den = sums[5];
            if (lane == 0) {
                const float4 old = L.x4[p];
                const float4 nw = make_float4(n0 / den, n1 / den, n2 / den, n3 / den);
                change = fabsf(nw.x - old.x) + fabsf(nw.y - old.y) + fabsf(nw.z - old.z);
                L.x4[p] = nw;
                if (C5)
                    L.x1[p] = n4 / den;
                if (L.h4)
                    shadow_store_raise(L, p, nw);
                if (a.hp)
                    a.hp[p] = 0;
            }
        }
        if (lane == 0)
            a.partials[item] = change;   // one value per voxel, summed in a fixed order
    }
}

template <bool C5>
__global__ void __launch_bounds__(VOTE_BLOCK, VOTE_MIN_BLOCKS) k_vote(const VoteArgs a)
{
    const int item = blockIdx.x * VOTE_WARPS + (threadIdx.x >> 5);
    if (item < a.n)
        vote_one<C5>(a, item, threadIdx.x & 31, vote_lane(threadIdx.x & 31));
}

// Batch form: warp g takes occluded voxel g of the clips' concatenated lists
// (clip c owns [prefix[c], prefix[c+1])), one voxel per warp as in k_vote. A
// data-sized grid: a persistent grid-stride form sized for 8 resident blocks
// per SM got 5 (46 registers), and its remaining blocks ran their whole share
// of the voxels as a late second wave.
template <bool C5>
__global__ void __launch_bounds__(VOTE_BLOCK, VOTE_MIN_BLOCKS) k_vote_batch(const BatchClip *__restrict__ clips,
                                                           const int *__restrict__ prefix, int n)
{
    const int g = blockIdx.x * VOTE_WARPS + (threadIdx.x >> 5);
    if (g >= __ldg(prefix + n))
        return;
    const int c = find_segment(prefix, n, g);
    vote_one<C5>(clips[c].vote, g - __ldg(prefix + c), threadIdx.x & 31, vote_lane(threadIdx.x & 31));
}

void launch_vote_batch(const BatchClip *clips, const int *hprefix, int n, int total_holes, bool c5,
                       cudaStream_t st)
{
    if (total_holes <= 0 || n <= 0)
        return;
    VI_COUNT_LAUNCH();
    const int grid = blocks_for(total_holes, VOTE_WARPS);
    if (c5)
        k_vote_batch<true><<<grid, VOTE_BLOCK, 0, st>>>(clips, hprefix, n);
    else
        k_vote_batch<false><<<grid, VOTE_BLOCK, 0, st>>>(clips, hprefix, n);
}

void launch_vote(const VoteArgs &a, bool c5, cudaStream_t st)
{
    if (a.n <= 0)
        return;
    VI_COUNT_LAUNCH();
    const int grid = blocks_for(a.n, VOTE_WARPS);   // one warp per voxel
    if (c5)
        k_vote<true><<<grid, VOTE_BLOCK, 0, st>>>(a);
    else
        k_vote<false><<<grid, VOTE_BLOCK, 0, st>>>(a);
}

// Deterministic sum of n values by one block of 256 threads: thread j adds
// elements j, j + 256, ... in FP64, then a fixed-order tree in shared
// memory. The result depends only on the values, not on where they sit.
template <typename T>
__device__ double block_sum_range(const T *__restrict__ v, int n)
{
    __shared__ double s[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += 256)
        acc += (double)v[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    const double r = s[0];
    __syncthreads();
    return r;
}

// The sum of a per-voxel array (the vote's changes, for e) in two stages that
// spread the FP64 work over the SMs (FP64 is slow on one SM): every chunk of
// SUM_CHUNK consecutive values, counted from the start of the clip's array,
// is summed by one block, then the chunk sums by one block, both with
// block_sum_range. The order depends only on the clip's own values, so a
// clip's e is the same alone (launch_sum_partials) and in a batch
// (launch_segment_sums).
static constexpr int SUM_CHUNK = 2048;

int sum_chunks(int n) { return n > 0 ? (n + SUM_CHUNK - 1) / SUM_CHUNK : 0; }

__global__ void k_chunk_sums(const float *__restrict__ vals, int n, double *__restrict__ chunks)
{
    const int lo = blockIdx.x * SUM_CHUNK;
    const double r = block_sum_range(vals + lo, min(SUM_CHUNK, n - lo));
    if (threadIdx.x == 0)
        chunks[blockIdx.x] = r;
}

__global__ void k_sum_chunks(const double *__restrict__ chunks, int nc, double *out)
{
    const double r = block_sum_range(chunks, nc);
    if (threadIdx.x == 0)
        out[0] = r;
}

void launch_sum_partials(const float *partials, int n, double *chunks, double *out, cudaStream_t st)
{
    const int nc = sum_chunks(n);
    if (nc > 0) {
        VI_COUNT_LAUNCH();
        k_chunk_sums<<<nc, 256, 0, st>>>(partials, n, chunks);
    }
    VI_COUNT_LAUNCH();
    k_sum_chunks<<<1, 256, 0, st>>>(chunks, nc, out);
}

// Batch form: segment i of vals is [starts[i], starts[i+1]); its chunks are
// chunks[cprefix[i] .. cprefix[i+1]).
__global__ void k_chunk_sums_batch(const float *__restrict__ vals, const int *__restrict__ starts,
                                   const int *__restrict__ cprefix, int nseg, double *__restrict__ chunks)
{
    const int b = blockIdx.x;
    const int seg = find_segment(cprefix, nseg, b);
    const int lo = starts[seg] + (b - cprefix[seg]) * SUM_CHUNK;
    const double r = block_sum_range(vals + lo, min(SUM_CHUNK, starts[seg + 1] - lo));
    if (threadIdx.x == 0)
        chunks[b] = r;
}

__global__ void k_segment_sums(const double *__restrict__ chunks, const int *__restrict__ cprefix, int nseg,
                               double *out)
{
    const int i = blockIdx.x;
    if (i >= nseg)
        return;
    const double r = block_sum_range(chunks + cprefix[i], cprefix[i + 1] - cprefix[i]);
    if (threadIdx.x == 0)
        out[i] = r;
}

void launch_segment_sums(const float *vals, const int *starts, const int *cprefix, int nseg, int total_chunks,
                         double *chunks, double *out, cudaStream_t st)
{
    if (nseg <= 0)
        return;
    if (total_chunks > 0) {
        VI_COUNT_LAUNCH();
        k_chunk_sums_batch<<<total_chunks, 256, 0, st>>>(vals, starts, cprefix, nseg, chunks);
    }
    VI_COUNT_LAUNCH();
    k_segment_sums<<<nseg, 256, 0, st>>>(chunks, cprefix, nseg, out);
}

// Eq. 6: the occluded voxel p copies u(p + phi(q*)), q* = argmin d2(q) over
// q in N_p inside the video, first in (dt, dy, dx) order on ties.
template <bool C5>
__global__ void k_final(LevelView L, const int *__restrict__ holes, int nH, const Shift *__restrict__ phi,
                        const float *__restrict__ d2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nH)
        return;
    const int p = holes[i];
    int px, py, pt;
    decode(p, L.W, L.HW, px, py, pt);
    float bd = 0.0f;
    int bq = -1;
    for (int dt = -2; dt <= 2; ++dt)
        for (int dy = -2; dy <= 2; ++dy)
            for (int dx = -2; dx <= 2; ++dx) {
                if (!inside(L, px + dx, py + dy, pt + dt))
                    continue;
                const int q = p + dt * L.HW + dy * L.W + dx;
                const float d = d2[q];
                if (bq < 0 || d < bd) {
                    bd = d;
                    bq = q;
                }
            }
    const Shift f = phi[bq];
    if (!inside(L, px + f.dx, py + f.dy, pt + f.dt))   // only for an invalid injected map
        return;
    const int s = p + (int)f.dt * L.HW + (int)f.dy * L.W + (int)f.dx;
    const float4 a = L.x4[s];
    L.x4[p] = a;
    if (C5)
        L.x1[p] = L.x1[s];
    if (L.h4)
        shadow_store_raise(L, p, a);
}

void launch_final(LevelView L, const int *holes, int nH, const Shift *phi, const float *d2, bool c5,
                  cudaStream_t st)
{
    if (nH <= 0)
        return;
    VI_COUNT_LAUNCH();
    if (c5)
        k_final<true><<<blocks_for(nH, 256), 256, 0, st>>>(L, holes, nH, phi, d2);
    else
        k_final<false><<<blocks_for(nH, 256), 256, 0, st>>>(L, holes, nH, phi, d2);
}

// Eq. 1: per-block sums of d^2 over H and over H~ (FP32 distances, FP64 sums).
int energy_blocks(int n) { return blocks_for(n, 256); }

template <bool C5>
__global__ void k_energy(LevelView L, const int *__restrict__ targets, int nT, const Shift *__restrict__ phi,
                         double *partials2)
{
    __shared__ double sh[2][256];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double eh = 0.0, et = 0.0;
    if (i < nT) {
        const int p = targets[i];
        int px, py, pt;
        decode(p, L.W, L.HW, px, py, pt);
        const Shift f = phi[p];
        const int sx = px + f.dx, sy = py + f.dy, st = pt + f.dt;
        double d = __longlong_as_double(0x7ff0000000000000ll);
        if (sx >= 2 && sx < L.W - 2 && sy >= 2 && sy < L.H - 2 && st >= 2 && st < L.T - 2)
            d = (double)patch_d2<C5>(L, p, px, py, pt, st * L.HW + sy * L.W + sx, nullptr);
        et = d;
        if (L.code[p] & CODE_HOLE)
            eh = d;
    }
    sh[0][threadIdx.x] = eh;
    sh[1][threadIdx.x] = et;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials2[2 * blockIdx.x] = sh[0][0];
        partials2[2 * blockIdx.x + 1] = sh[1][0];
    }
}

void launch_energy(LevelView L, const int *targets, int nT, const Shift *phi, bool c5, double *partials2,
                   cudaStream_t st)
{
    if (nT <= 0)
        return;
    VI_COUNT_LAUNCH();
    if (c5)
        k_energy<true><<<energy_blocks(nT), 256, 0, st>>>(L, targets, nT, phi, partials2);
    else
        k_energy<false><<<energy_blocks(nT), 256, 0, st>>>(L, targets, nT, phi, partials2);
}

__global__ void k_sum_partials2(const double *__restrict__ p2, int n, double *out2)
{
    __shared__ double s[2][256];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) {
        a += p2[2 * i];
        b += p2[2 * i + 1];
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s[0][threadIdx.x] += s[0][threadIdx.x + o];
            s[1][threadIdx.x] += s[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out2[0] = s[0][0];
        out2[1] = s[1][0];
    }
}

void launch_sum_partials2(const double *partials2, int n, double *out2, cudaStream_t st)
{
    VI_COUNT_LAUNCH();
    k_sum_partials2<<<1, 256, 0, st>>>(partials2, n, out2);
}

// Algorithm 3 sets. layer = H' minus its 3x3x3 erosion (voxels outside the
// video are not in H'); ltgt = voxels outside H' whose patch meets the layer.
__global__ void k_onion_layer(LevelView L, const uint8_t *__restrict__ hp, uint8_t *__restrict__ layer)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < L.V;
         v += (long long)gridDim.x * blockDim.x) {
        uint8_t out = 0;
        if (hp[v]) {
            int x, y, t;
            decode((int)v, L.W, L.HW, x, y, t);
            bool all = true;
            for (int dt = -1; dt <= 1 && all; ++dt)
                for (int dy = -1; dy <= 1 && all; ++dy)
                    for (int dx = -1; dx <= 1 && all; ++dx) {
                        if (!inside(L, x + dx, y + dy, t + dt) ||
                            !hp[(t + dt) * L.HW + (y + dy) * L.W + x + dx])
                            all = false;
                    }
            out = all ? 0 : 1;
        }
        layer[v] = out;
    }
}

void launch_onion_layer(LevelView L, const uint8_t *hp, uint8_t *layer, cudaStream_t st)
{
    VI_COUNT_LAUNCH();
    k_onion_layer<<<blocks_for(L.V, 256), 256, 0, st>>>(L, hp, layer);
}

__global__ void k_onion_targets(LevelView L, const uint8_t *__restrict__ hp, const uint8_t *__restrict__ layer,
                                uint8_t *__restrict__ ltgt)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < L.V;
         v += (long long)gridDim.x * blockDim.x) {
        uint8_t out = 0;
        if (!hp[v]) {
            int x, y, t;
            decode((int)v, L.W, L.HW, x, y, t);
            for (int dt = -2; dt <= 2 && !out; ++dt)
                for (int dy = -2; dy <= 2 && !out; ++dy)
                    for (int dx = -2; dx <= 2 && !out; ++dx)
                        if (inside(L, x + dx, y + dy, t + dt) &&
                            layer[(t + dt) * L.HW + (y + dy) * L.W + x + dx])
                            out = 1;
        }
        ltgt[v] = out;
    }
}

void launch_onion_targets(LevelView L, const uint8_t *hp, const uint8_t *layer, uint8_t *ltgt,
                          cudaStream_t st)
{
    VI_COUNT_LAUNCH();
    k_onion_targets<<<blocks_for(L.V, 256), 256, 0, st>>>(L, hp, layer, ltgt);
}

__global__ void k_count(const uint8_t *__restrict__ flags, int V, int *count)
{
    int c = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x)
        c += flags[v] ? 1 : 0;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c)
        atomicAdd(count, c);
}

void launch_count(const uint8_t *flags, int V, int *count_dev, cudaStream_t st)
{
    cudaMemsetAsync(count_dev, 0, sizeof(int), st);
    int g = blocks_for(V, 256);
    if (g > 152 * 8)
        g = 152 * 8;
    VI_COUNT_LAUNCH();
    k_count<<<g, 256, 0, st>>>(flags, V, count_dev);
}

// Layout packing: [V] float4 (+ float) <-> [V][C] float32.
// One output float per thread, so that a warp writes 128 consecutive bytes:
// the destination may be pinned host memory written across the chip-to-chip
// link, where whole lines matter (three threads read each source voxel, from
// L1).
__global__ void k_pack_rgb(LevelView L, float *__restrict__ rgb)
{
    const long long n = 3ll * L.V;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n;
         o += (long long)gridDim.x * blockDim.x) {
        const long long v = o / 3;
        const int c = (int)(o - 3 * v);
        const float *a = reinterpret_cast<const float *>(L.x4 + v);
        rgb[o] = a[c];
    }
}

void launch_pack_rgb(LevelView L, float *rgb, cudaStream_t st)
{
    long long g = (3ll * L.V + 255) / 256;
    if (g > 152 * 16)
        g = 152 * 16;
    if (g < 1)
        g = 1;
    VI_COUNT_LAUNCH();
    k_pack_rgb<<<(int)g, 256, 0, st>>>(L, rgb);
}

// dst[0 .. n) = src[0 .. n): 16 bytes per thread and iteration when both
// addresses are 16-byte aligned, else single bytes. src may be pinned host
// memory read across the chip-to-chip link: many loads in flight, rather than
// the copy engine's one stream of page translations.
__global__ void k_copy_bytes(uint8_t *__restrict__ dst, const uint8_t *__restrict__ src, long long n, bool wide)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long done = 0;
    if (wide) {
        const long long n16 = n / 16;
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst);
        for (long long i = t0; i < n16; i += stride)
            d4[i] = s4[i];
        done = n16 * 16;
    }
    for (long long i = done + t0; i < n; i += stride)
        dst[i] = src[i];
}

void launch_copy_bytes(void *dst, const void *src, long long n, cudaStream_t st)
{
    if (n <= 0)
        return;
    const bool wide = ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15u) == 0;
    long long g = (wide ? n / 16 : n) / 256 + 1;
    if (g > 152 * 16)
        g = 152 * 16;
    VI_COUNT_LAUNCH();
    k_copy_bytes<<<(int)g, 256, 0, st>>>(static_cast<uint8_t *>(dst), static_cast<const uint8_t *>(src), n, wide);
}

// The channels of list[0 .. n) packed into buf4[0 .. n) (c0..c3) and
// buf1[0 .. n) (c4), or (unpack) written back from there.
__global__ void k_pack_voxels(LevelView L, const int *__restrict__ list, int n, float4 *buf4, float *buf1,
                              bool unpack)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int v = list[i];
        if (unpack) {
            L.x4[v] = buf4[i];
            if (L.x1)
                L.x1[v] = buf1[i];
        } else {
            buf4[i] = L.x4[v];
            if (L.x1)
                buf1[i] = L.x1[v];
        }
    }
}

void launch_pack_voxels(LevelView L, const int *list, int n, float4 *buf4, float *buf1, bool unpack,
                        cudaStream_t st)
{
    if (n <= 0)
        return;
    VI_COUNT_LAUNCH();
    k_pack_voxels<<<blocks_for(n, 256), 256, 0, st>>>(L, list, n, buf4, buf1, unpack);
}

__global__ void k_get_channels(LevelView L, float *__restrict__ out, int C)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < L.V;
         v += (long long)gridDim.x * blockDim.x) {
        const float4 a = L.x4[v];
        out[C * v] = a.x;
        out[C * v + 1] = a.y;
        out[C * v + 2] = a.z;
        if (C == 5) {
            out[C * v + 3] = a.w;
            out[C * v + 4] = L.x1[v];
        }
    }
}

void launch_get_channels(LevelView L, float *out, int C, cudaStream_t st)
{
    VI_COUNT_LAUNCH();
    k_get_channels<<<blocks_for(L.V, 256), 256, 0, st>>>(L, out, C);
}

__global__ void k_set_channels(LevelView L, const float *__restrict__ in, int C)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < L.V;
         v += (long long)gridDim.x * blockDim.x) {
        float4 a = make_float4(in[C * v], in[C * v + 1], in[C * v + 2], 0.0f);
        if (C == 5) {
            a.w = in[C * v + 3];
            L.x1[v] = in[C * v + 4];
        }
        L.x4[v] = a;
    }
}

void launch_set_channels(LevelView L, const float *in, int C, cudaStream_t st)
{
    VI_COUNT_LAUNCH();
    k_set_channels<<<blocks_for(L.V, 256), 256, 0, st>>>(L, in, C);
}

// FP16 copies of every voxel of a level; hmax raised once per warp.
__global__ void k_shadow_all(LevelView L)
{
    unsigned m0 = 0, m1 = 0, m2 = 0, m3 = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < L.V; v += gridDim.x * blockDim.x) {
        const float4 a = L.x4[v];
        shadow_store(L, v, a);
        m0 = max(m0, abs_bits(a.x));
        m1 = max(m1, abs_bits(a.y));
        m2 = max(m2, abs_bits(a.z));
        m3 = max(m3, abs_bits(a.w));
    }
    m0 = __reduce_max_sync(0xffffffffu, m0);
    m1 = __reduce_max_sync(0xffffffffu, m1);
    m2 = __reduce_max_sync(0xffffffffu, m2);
    m3 = __reduce_max_sync(0xffffffffu, m3);
    if ((threadIdx.x & 31) == 0) {
        raise_hmax(L.hmax, 0, m0);
        raise_hmax(L.hmax, 1, m1);
        raise_hmax(L.hmax, 2, m2);
        raise_hmax(L.hmax, 3, m3);
    }
}

void launch_shadow_all(LevelView L, cudaStream_t st)
{
    if (!L.h4 || L.V <= 0)
        return;
    long long g = ((long long)L.V + 255) / 256;
    if (g > 152 * 16)
        g = 152 * 16;
    VI_COUNT_LAUNCH();
    k_shadow_all<<<(int)g, 256, 0, st>>>(L);
}

}  // namespace vi

namespace vi {

__global__ void k_extract_bit(const uint8_t *__restrict__ in, uint8_t bit, uint8_t *__restrict__ out, int V)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x)
        out[v] = (in[v] & bit) ? 1 : 0;
}

void launch_extract_bit(const uint8_t *in, uint8_t bit, uint8_t *out, int V, cudaStream_t st)
{
    VI_COUNT_LAUNCH();
    k_extract_bit<<<blocks_for(V, 256), 256, 0, st>>>(in, bit, out, V);
}

__global__ void k_fill_f32(float *__restrict__ dst, float value, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = value;
}

void launch_fill_f32(float *dst, float value, long long n, cudaStream_t st)
{
    long long g = (n + 255) / 256;
    if (g > 152 * 16)
        g = 152 * 16;
    if (g < 1)
        g = 1;
    VI_COUNT_LAUNCH();
    k_fill_f32<<<(int)g, 256, 0, st>>>(dst, value, n);
}

}  // namespace vi
