// vi_pyramid.cu -- Algorithm 4's pyramid construction: texture features at full
// resolution (Eq. 7), colour / occlusion pyramids (Sec. 3.6), texture pyramid
// by subsampling (Eq. 8), the sets H~ and D~ of Sec. 2 and their voxel lists.
//
// All kernels are one thread per output voxel over a grid-stride loop: this
// stage is a single HBM pass per level, far below 1% of a run.
#include "vi_launch.h"

namespace vi {

static inline int grid_for(long long n, int block)
{
    long long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (int)g;
}

// ---------------------------------------------------------------------------
// Eq. 7: grey level I = (R + G + B) / 3; I_x, I_y central differences, one-sided
// on the frame border; a sample is known when its two stencil voxels are.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float grey(const float *rgb, long long v)
{
    return (rgb[3 * v] + rgb[3 * v + 1] + rgb[3 * v + 2]) / 3.0f;
}

__global__ void k_gradients(const float *__restrict__ rgb, const uint8_t *__restrict__ hole, int W,
                            int H, int T, float2 *__restrict__ g, uint8_t *__restrict__ valid)
{
    const long long V = (long long)W * H * T;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
         v += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(v % W);
        const int y = (int)((v / W) % H);
        const long long row = v - x;        // voxel (0, y, t)
        const long long col = v - (long long)y * W;  // voxel (x, 0, t)
        float gx = 0.0f, gy = 0.0f;
        uint8_t ok = 0;
        if (W >= 2) {
            int a, b;
            float den;
            if (x == 0) { a = 0; b = 1; den = 1.0f; }
            else if (x == W - 1) { a = W - 2; b = W - 1; den = 1.0f; }
            else { a = x - 1; b = x + 1; den = 2.0f; }
            if (!hole[row + a] && !hole[row + b]) {
                gx = fabsf((grey(rgb, row + b) - grey(rgb, row + a)) / den);
                ok |= 1;
            }
        }
        if (H >= 2) {
            int a, b;
            float den;
            if (y == 0) { a = 0; b = 1; den = 1.0f; }
            else if (y == H - 1) { a = H - 2; b = H - 1; den = 1.0f; }
            else { a = y - 1; b = y + 1; den = 2.0f; }
            if (!hole[col + (long long)a * W] && !hole[col + (long long)b * W]) {
                gy = fabsf((grey(rgb, col + (long long)b * W) - grey(rgb, col + (long long)a * W)) / den);
                ok |= 2;
            }
        }
        g[v] = make_float2(gx, gy);
        valid[v] = ok;
    }
}

void launch_gradients(const float *rgb, const uint8_t *hole, int W, int H, int T, float2 *g,
                      uint8_t *valid, cudaStream_t st)
{
    VI_COUNT_LAUNCH();
    k_gradients<<<grid_for((long long)W * H * T, 256), 256, 0, st>>>(rgb, hole, W, H, T, g, valid);
}

// Separable box over nu = offsets [lo, lo + side - 1] in x then in y, keeping
// sums and counts of known samples; T = sum / count (0 with no known sample).
__global__ void k_box_x(const float2 *__restrict__ g, const uint8_t *__restrict__ valid, int W, int H,
                        int T, int lo, int side, float2 *__restrict__ sum, uint16_t *__restrict__ cnt)
{
    const long long V = (long long)W * H * T;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
         v += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(v % W);
        const long long row = v - x;
        float sx = 0.0f, sy = 0.0f;
        int nx = 0, ny = 0;
        for (int i = 0; i < side; ++i) {
            const int qx = x + lo + i;
            if (qx < 0 || qx >= W)
                continue;
            const uint8_t ok = valid[row + qx];
            const float2 gg = g[row + qx];
            if (ok & 1) { sx += gg.x; ++nx; }
            if (ok & 2) { sy += gg.y; ++ny; }
        }
        sum[v] = make_float2(sx, sy);
        cnt[2 * v] = (uint16_t)nx;
        cnt[2 * v + 1] = (uint16_t)ny;
    }
}

__global__ void k_box_y(const float2 *__restrict__ sum, const uint16_t *__restrict__ cnt, int W,
                        int H, int T, int lo, int side, float2 *__restrict__ T0)
{
    const long long V = (long long)W * H * T;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
         v += (long long)gridDim.x * blockDim.x) {
        const int y = (int)((v / W) % H);
        const long long col = v - (long long)y * W;
        float sx = 0.0f, sy = 0.0f;
        int nx = 0, ny = 0;
        for (int j = 0; j < side; ++j) {
            const int qy = y + lo + j;
            if (qy < 0 || qy >= H)
                continue;
            const long long q = col + (long long)qy * W;
            const float2 s = sum[q];
            sx += s.x;
            sy += s.y;
            nx += cnt[2 * q];
            ny += cnt[2 * q + 1];
        }
        T0[v] = make_float2(nx ? sx / (float)nx : 0.0f, ny ? sy / (float)ny : 0.0f);
    }
}

void launch_box_mean(const float2 *g, const uint8_t *valid, int W, int H, int T, int side,
                     float2 *tmp_sum, uint16_t *tmp_cnt, float2 *T0, cudaStream_t st)
{
    const int lo = -(side / 2);
    const int grid = grid_for((long long)W * H * T, 256);
    VI_COUNT_LAUNCH();
    k_box_x<<<grid, 256, 0, st>>>(g, valid, W, H, T, lo, side, tmp_sum, tmp_cnt);
    VI_COUNT_LAUNCH();
    k_box_y<<<grid, 256, 0, st>>>(tmp_sum, tmp_cnt, W, H, T, lo, side, T0);
}

__global__ void k_level0_channels(const float *__restrict__ rgb, const uint8_t *__restrict__ hole,
                                  const float2 *__restrict__ T0, float s, int c5, LevelView L)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < L.V;
         v += (long long)gridDim.x * blockDim.x) {
        const bool h = hole[v] != 0;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        float b = 0.0f;
        if (!h) {
            a.x = rgb[3 * v];
            a.y = rgb[3 * v + 1];
            a.z = rgb[3 * v + 2];
            if (c5) {
                const float2 t = T0[v];
                a.w = s * t.x;
                b = s * t.y;
            }
        }
        L.x4[v] = a;
        if (c5)
            L.x1[v] = b;
        L.code[v] = h ? CODE_HOLE : 0;
    }
}

void launch_level0_channels(const float *rgb, const uint8_t *hole, const float2 *T0,
                            float sqrt_lambda, bool c5, LevelView L, cudaStream_t st)
{
    VI_COUNT_LAUNCH();
    k_level0_channels<<<grid_for(L.V, 256), 256, 0, st>>>(rgb, hole, T0, sqrt_lambda, c5 ? 1 : 0, L);
}

// Colour / occlusion pyramid step and Eq. 8 subsampling of the features:
// 2x2 children of the same frame, or with tsub (the temporal subsampling
// option) 2x2x2 children of frames 2t, 2t+1, the features then sampled at
// frame 2^level t.
__global__ void k_downsample(LevelView F, LevelView Cs, int level, const float2 *__restrict__ T0,
                             int W0, int H0, float s, int c5, int tsub)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < Cs.V;
         v += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(v % Cs.W);
        const int y = (int)((v / Cs.W) % Cs.H);
        const int t = (int)(v / Cs.HW);
        bool occl = false;
        int n = 0;
        float r = 0.f, g = 0.f, b = 0.f;
        for (int k = 0; k <= tsub; ++k)
            for (int j = 0; j < 2; ++j)
                for (int i = 0; i < 2; ++i) {
                    const int fx = 2 * x + i, fy = 2 * y + j, ft = tsub ? 2 * t + k : t;
                    if (fx >= F.W || fy >= F.H || ft >= F.T)
                        continue;
                    const long long f = (long long)ft * F.HW + (long long)fy * F.W + fx;
                    if (F.code[f] & CODE_HOLE)
                        occl = true;
                    const float4 a = F.x4[f];
                    r += a.x; g += a.y; b += a.z;
                    ++n;
                }
        float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
        float o1 = 0.0f;
        if (!occl) {
            out.x = r / (float)n;
            out.y = g / (float)n;
            out.z = b / (float)n;
            if (c5) {
                const int t0 = tsub ? (t << level) : t;
                const long long q = (long long)t0 * W0 * H0 + (long long)(y << level) * W0 + (x << level);
                const float2 tq = T0[q];
                out.w = s * tq.x;
                o1 = s * tq.y;
            }
        }
        Cs.x4[v] = out;
        if (c5)
            Cs.x1[v] = o1;
        Cs.code[v] = occl ? CODE_HOLE : 0;
    }
}

void launch_downsample(LevelView fine, LevelView coarse, int level, const float2 *T0, int W0, int H0,
                       float sqrt_lambda, bool c5, bool tsub, cudaStream_t st)
{
    VI_COUNT_LAUNCH();
    k_downsample<<<grid_for(coarse.V, 256), 256, 0, st>>>(fine, coarse, level, T0, W0, H0,
                                                           sqrt_lambda, c5 ? 1 : 0, tsub ? 1 : 0);
}

// ---------------------------------------------------------------------------
// H~ = dilation of H by the 5x5x5 box (clipped to the video); D~ = voxels
// whose patch is inside the video and misses H, i.e. interior and not in the
// dilation. Three separable passes of a radius-2 OR along x, y, t.
// ---------------------------------------------------------------------------
__global__ void k_dilate_axis(const uint8_t *__restrict__ src, uint8_t srcbit, uint8_t *__restrict__ dst,
                              int W, int H, int T, int axis)
{
    const long long V = (long long)W * H * T;
    const long long HW = (long long)W * H;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
         v += (long long)gridDim.x * blockDim.x) {
        int c, n;
        long long stride;
        if (axis == 0) { c = (int)(v % W); n = W; stride = 1; }
        else if (axis == 1) { c = (int)((v / W) % H); n = H; stride = W; }
        else { c = (int)(v / HW); n = T; stride = HW; }
        uint8_t any = 0;
        for (int d = -2; d <= 2; ++d) {
            const int q = c + d;
            if (q < 0 || q >= n)
                continue;
            if (src[v + d * stride] & srcbit)
                any = 1;
        }
        dst[v] = any;
    }
}

__global__ void k_codes(LevelView L, const uint8_t *__restrict__ near)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < L.V;
         v += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(v % L.W);
        const int y = (int)((v / L.W) % L.H);
        const int t = (int)(v / L.HW);
        const bool interior = x >= 2 && x < L.W - 2 && y >= 2 && y < L.H - 2 && t >= 2 && t < L.T - 2;
        uint8_t c = L.code[v] & CODE_HOLE;
        if (near[v])
            c |= CODE_TARGET;
        else if (interior)
            c |= CODE_SOURCE;
        L.code[v] = c;
    }
}

// Bounding box of the occluded pixels of every frame, for the level rule of
// Sec. 3.6: out[t] = (x0, x1, y0, y1), or (W, -1, H, -1) for a frame without
// one. One block per frame; the threads scan its pixels, then warp and block
// reductions.
__global__ void __launch_bounds__(512) k_mask_extents(const uint8_t *__restrict__ mask, int W, int H,
                                                     int4 *__restrict__ out)
{
    const unsigned FULL = 0xffffffffu;
    const uint8_t *m = mask + (size_t)blockIdx.x * W * H;
    const int n = W * H;
    int x0 = W, x1 = -1, y0 = H, y1 = -1;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        if (m[i]) {
            const int y = i / W, x = i - y * W;
            x0 = min(x0, x);
            x1 = max(x1, x);
            y0 = min(y0, y);
            y1 = max(y1, y);
        }
    x0 = __reduce_min_sync(FULL, x0);
    x1 = __reduce_max_sync(FULL, x1);
    y0 = __reduce_min_sync(FULL, y0);
    y1 = __reduce_max_sync(FULL, y1);
    __shared__ int4 part[16];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        part[warp] = make_int4(x0, x1, y0, y1);
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        const int4 v = lane < nw ? part[lane] : make_int4(W, -1, H, -1);
        const int a = __reduce_min_sync(FULL, v.x), b = __reduce_max_sync(FULL, v.y),
                  c = __reduce_min_sync(FULL, v.z), d = __reduce_max_sync(FULL, v.w);
        if (lane == 0)
            out[blockIdx.x] = make_int4(a, b, c, d);
    }
}

void launch_mask_extents(const uint8_t *mask, int W, int H, int T, int4 *out, cudaStream_t st)
{
    VI_COUNT_LAUNCH();
    k_mask_extents<<<T, 512, 0, st>>>(mask, W, H, out);
}

void launch_codes(LevelView L, uint8_t *tmp_a, uint8_t *tmp_b, cudaStream_t st)
{
    const int grid = grid_for(L.V, 256);
    VI_COUNT_LAUNCH();
    k_dilate_axis<<<grid, 256, 0, st>>>(L.code, CODE_HOLE, tmp_a, L.W, L.H, L.T, 0);
    VI_COUNT_LAUNCH();
    k_dilate_axis<<<grid, 256, 0, st>>>(tmp_a, 1, tmp_b, L.W, L.H, L.T, 1);
    VI_COUNT_LAUNCH();
    k_dilate_axis<<<grid, 256, 0, st>>>(tmp_b, 1, tmp_a, L.W, L.H, L.T, 2);
    VI_COUNT_LAUNCH();
    k_codes<<<grid, 256, 0, st>>>(L, tmp_a);
}

// ---------------------------------------------------------------------------
// Stream compaction in raster order: per-block counts, one-block scan, write.
// ---------------------------------------------------------------------------
static constexpr int CB = 1024;  // voxels per compaction block (one per thread)

int compact_blocks(int V) { return (V + CB - 1) / CB; }

__global__ void k_compact_count(const uint8_t *__restrict__ flags, uint8_t bits, int V, int *counts)
{
    const int v = blockIdx.x * CB + threadIdx.x;
    const int f = (v < V && (flags[v] & bits)) ? 1 : 0;
    const int c = __syncthreads_count(f);
    if (threadIdx.x == 0)
        counts[blockIdx.x] = c;
}

// Exclusive scan of counts[0..nb) in place; counts[nb] and *total get the sum.
// Block j of the grid scans the array at counts + j * stride into total[j].
__global__ void k_compact_scan(int *counts, int nb, int *total, int stride)
{
    counts += blockIdx.x * stride;
    total += blockIdx.x;
    __shared__ int warp_tot[32];
    __shared__ int carry;
    if (threadIdx.x == 0)
        carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < nb ? counts[i] : 0;
        // inclusive warp scan
        int s = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, s, o);
            if ((threadIdx.x & 31) >= o)
                s += t;
        }
        if ((threadIdx.x & 31) == 31)
            warp_tot[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x < 32) {
            int w = warp_tot[threadIdx.x];
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, w, o);
                if (threadIdx.x >= o)
                    w += t;
            }
            warp_tot[threadIdx.x] = w;   // inclusive over warps
        }
        __syncthreads();
        const int wid = threadIdx.x >> 5;
        const int excl = s - v + (wid ? warp_tot[wid - 1] : 0) + carry;
        if (i < nb)
            counts[i] = excl;
        __syncthreads();
        if (threadIdx.x == 1023)
            carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        counts[nb] = carry;
        *total = carry;
    }
}

__global__ void k_compact_write(const uint8_t *__restrict__ flags, uint8_t bits, int V,
                                const int *__restrict__ offsets, int *__restrict__ list)
{
    __shared__ int warp_cnt[CB / 32];
    const int v = blockIdx.x * CB + threadIdx.x;
    const int f = (v < V && (flags[v] & bits)) ? 1 : 0;
    const unsigned ballot = __ballot_sync(0xffffffffu, f);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
        warp_cnt[wid] = __popc(ballot);
    __syncthreads();
    if (f) {
        int before = 0;
        for (int w = 0; w < wid; ++w)
            before += warp_cnt[w];
        before += __popc(ballot & ((1u << lane) - 1u));
        list[offsets[blockIdx.x] + before] = v;
    }
}

void launch_compact(const uint8_t *flags, uint8_t bits, int V, int *block_counts, int *list,
                    int *count_dev, cudaStream_t st)
{
    const int nb = compact_blocks(V);
    VI_COUNT_LAUNCH();
    k_compact_count<<<nb, CB, 0, st>>>(flags, bits, V, block_counts);
    VI_COUNT_LAUNCH();
    k_compact_scan<<<1, 1024, 0, st>>>(block_counts, nb, count_dev, 0);
    VI_COUNT_LAUNCH();
    if (list)
        k_compact_write<<<nb, CB, 0, st>>>(flags, bits, V, block_counts, list);
}

// The three lists of a level's set codes at once (bits b.x, b.y, b.z of
// flags): one pass counts all three per block (counts j at
// block_counts[j * (nb + 1) ..]), one launch scans the three arrays (sizes to
// count_dev[0..2]), and after the caller has read the sizes and allocated
// the lists, one pass writes all three, raster ordered, from the same
// offsets.
__global__ void k_compact_count3(const uint8_t *__restrict__ flags, uchar3 b, int V, int nb, int *counts)
{
    const int v = blockIdx.x * CB + threadIdx.x;
    const unsigned f = v < V ? flags[v] : 0u;
    const int c0 = __syncthreads_count(f & b.x);
    const int c1 = __syncthreads_count(f & b.y);
    const int c2 = __syncthreads_count(f & b.z);
    if (threadIdx.x == 0) {
        counts[blockIdx.x] = c0;
        counts[(nb + 1) + blockIdx.x] = c1;
        counts[2 * (nb + 1) + blockIdx.x] = c2;
    }
}

__global__ void k_compact_write3(const uint8_t *__restrict__ flags, uchar3 b, int V, int nb,
                                 const int *__restrict__ offsets, int *__restrict__ l0, int *__restrict__ l1,
                                 int *__restrict__ l2)
{
    __shared__ int warp_cnt[3][CB / 32];
    const int v = blockIdx.x * CB + threadIdx.x;
    const unsigned f = v < V ? flags[v] : 0u;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned bits[3] = {b.x, b.y, b.z};
    unsigned ballot[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        ballot[j] = __ballot_sync(0xffffffffu, (f & bits[j]) != 0u);
        if (lane == 0)
            warp_cnt[j][wid] = __popc(ballot[j]);
    }
    __syncthreads();
    int *lists[3] = {l0, l1, l2};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (f & bits[j]) {
            int before = 0;
            for (int w = 0; w < wid; ++w)
                before += warp_cnt[j][w];
            before += __popc(ballot[j] & ((1u << lane) - 1u));
            lists[j][offsets[j * (nb + 1) + blockIdx.x] + before] = v;
        }
    }
}

void launch_compact3_count(const uint8_t *flags, uchar3 bits, int V, int *block_counts, int *count_dev,
                           cudaStream_t st)
{
    const int nb = compact_blocks(V);
    VI_COUNT_LAUNCH();
    k_compact_count3<<<nb, CB, 0, st>>>(flags, bits, V, nb, block_counts);
    VI_COUNT_LAUNCH();
    k_compact_scan<<<3, 1024, 0, st>>>(block_counts, nb, count_dev, nb + 1);
}

void launch_compact3_write(const uint8_t *flags, uchar3 bits, int V, const int *block_counts, int *l0, int *l1,
                           int *l2, cudaStream_t st)
{
    const int nb = compact_blocks(V);
    VI_COUNT_LAUNCH();
    k_compact_write3<<<nb, CB, 0, st>>>(flags, bits, V, nb, block_counts, l0, l1, l2);
}

}  // namespace vi
