// vi_realign.cu -- the affine realignment of Sec. 3.4 (Algorithm 2,
// AlignVideo) and the UnwarpVideo step that ends Algorithm 4.
//
// EstimateAffineMotion is the robust fit of the dominant affine motion
// between successive frames (the paper cites Odobez and Bouthemy for it):
// Gauss-Newton on the six parameters of w(p) = (a0 + a1 x + a2 y,
// a3 + a4 x + a5 y) with iteratively reweighted least squares (Tukey's
// biweight, c = 4.6851 sigma, sigma^2 the weighted residual variance of the
// previous iteration, plain least squares first), over a 2x2 mean pyramid of
// the grey level (R + G + B) / 3 of the known pixels, coarse to fine. Every
// frame pair advances together: one launch per iteration accumulates the
// normal equations of all pairs (FP32 per pixel, FP64 across pixels in a
// fixed order), the host solves the 6x6 systems in double.
//
// Sample positions are computed in double without contraction (explicit
// round-to-nearest operations in the order (m0 x + m1 y) + m2), so whether a
// sample falls outside the frame or touches an occluded pixel is decided
// exactly as in double arithmetic; only the interpolated values are FP32.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "vi.h"
#include "vi_launch.h"

namespace vi {
namespace {

thread_local std::string g_realign_err;

vi_status rfail(vi_status st, const std::string &msg)
{
    g_realign_err = msg;
    return st;
}

#define RCK(call)                                                                                 \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return rfail(VI_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));        \
    } while (0)

constexpr double TUKEY_C = 4.6851;
constexpr double SIGMA_FLOOR = 1e-4;
constexpr int NRED = 29;          // 21 (upper triangle of J J^T) + 6 (J r) + sum w r^2 + sum w
constexpr int PIX_PER_THREAD = 8;

// ---- affine maps: 2x3 matrices, the same operation order as the host ----
struct Aff {
    double m[6];   // m00 m01 m02 m10 m11 m12
};

Aff from_theta(const double *a)
{
    Aff r;
    r.m[0] = 1.0 + a[1];
    r.m[1] = a[2];
    r.m[2] = a[0];
    r.m[3] = a[4];
    r.m[4] = 1.0 + a[5];
    r.m[5] = a[3];
    return r;
}

void to_theta(const Aff &m, double *a)
{
    a[0] = m.m[2];
    a[1] = m.m[0] - 1.0;
    a[2] = m.m[1];
    a[3] = m.m[5];
    a[4] = m.m[3];
    a[5] = m.m[4] - 1.0;
}

Aff compose(const Aff &b, const Aff &a)   // p -> b(a(p))
{
    Aff r;
    r.m[0] = b.m[0] * a.m[0] + b.m[1] * a.m[3];
    r.m[1] = b.m[0] * a.m[1] + b.m[1] * a.m[4];
    r.m[2] = b.m[0] * a.m[2] + b.m[1] * a.m[5] + b.m[2];
    r.m[3] = b.m[3] * a.m[0] + b.m[4] * a.m[3];
    r.m[4] = b.m[3] * a.m[1] + b.m[4] * a.m[4];
    r.m[5] = b.m[3] * a.m[2] + b.m[4] * a.m[5] + b.m[5];
    return r;
}

Aff invert(const Aff &a)
{
    const double det = a.m[0] * a.m[4] - a.m[1] * a.m[3];
    Aff r;
    r.m[0] = a.m[4] / det;
    r.m[1] = -a.m[1] / det;
    r.m[3] = -a.m[3] / det;
    r.m[4] = a.m[0] / det;
    r.m[2] = -(r.m[0] * a.m[2] + r.m[1] * a.m[5]);
    r.m[5] = -(r.m[3] * a.m[2] + r.m[4] * a.m[5]);
    return r;
}

// ---- device helpers -----------------------------------------------------------
__device__ __forceinline__ void affine_apply(const double *m, double x, double y, double &qx, double &qy)
{
    qx = __dadd_rn(__dadd_rn(__dmul_rn(m[0], x), __dmul_rn(m[1], y)), m[2]);
    qy = __dadd_rn(__dadd_rn(__dmul_rn(m[3], x), __dmul_rn(m[4], y)), m[5]);
}

// Bilinear sample set-up at (qx, qy) in [0, W-1] x [0, H-1].
struct Tap {
    int i00, i01, i10, i11;   // indices (x0,y0) (x1,y0) (x0,y1) (x1,y1)
    float fx, fy;
    bool ux, uy;              // x1 / y1 have a non-zero weight
};

__device__ __forceinline__ Tap make_tap(double qx, double qy, int W, int H)
{
    const double fxd = floor(qx), fyd = floor(qy);
    int x0 = (int)fxd, y0 = (int)fyd;
    const double ex = qx - fxd, ey = qy - fyd;
    x0 = min(max(x0, 0), W - 1);
    y0 = min(max(y0, 0), H - 1);
    const int x1 = min(x0 + 1, W - 1), y1 = min(y0 + 1, H - 1);
    Tap t;
    t.i00 = y0 * W + x0;
    t.i01 = y0 * W + x1;
    t.i10 = y1 * W + x0;
    t.i11 = y1 * W + x1;
    t.fx = (float)ex;
    t.fy = (float)ey;
    t.ux = ex > 0.0;
    t.uy = ey > 0.0;
    return t;
}

__device__ __forceinline__ float tap_value(const float *img, const Tap &t, int stride = 1, int c = 0)
{
    const float a = img[t.i00 * stride + c], b = img[t.i01 * stride + c];
    const float d = img[t.i10 * stride + c], e = img[t.i11 * stride + c];
    return (1.0f - t.fy) * ((1.0f - t.fx) * a + t.fx * b) + t.fy * ((1.0f - t.fx) * d + t.fx * e);
}

__device__ __forceinline__ bool tap_touches(const uint8_t *occ, const Tap &t)
{
    return occ[t.i00] || (t.ux && occ[t.i01]) || (t.uy && occ[t.i10]) || (t.ux && t.uy && occ[t.i11]);
}

// ---- pyramid of the grey level ------------------------------------------------
__global__ void k_grey(const float *__restrict__ rgb, const uint8_t *__restrict__ mask, long long n,
                       float *__restrict__ I, uint8_t *__restrict__ occ)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        I[i] = (rgb[3 * i] + rgb[3 * i + 1] + rgb[3 * i + 2]) / 3.0f;
        occ[i] = mask[i] ? 1 : 0;
    }
}

// 2x2 mean of the known children (sizes rounded up), occlusion by OR; T frames.
__global__ void k_grey_down(const float *__restrict__ I, const uint8_t *__restrict__ o, int W, int H, int T,
                            float *__restrict__ Ic, uint8_t *__restrict__ oc, int w, int h)
{
    const long long n = (long long)w * h * T;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int t = (int)(i / ((long long)w * h));
        const int r = (int)(i - (long long)t * w * h);
        const int y = r / w, x = r - y * w;
        float s = 0.0f;
        int cnt = 0;
        uint8_t oo = 0;
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                const int X = 2 * x + dx, Y = 2 * y + dy;
                if (X >= W || Y >= H)
                    continue;
                const long long j = ((long long)t * H + Y) * W + X;
                if (o[j])
                    oo = 1;
                else {
                    s += I[j];
                    ++cnt;
                }
            }
        Ic[i] = cnt ? s / (float)cnt : 0.0f;
        oc[i] = oo;
    }
}

// Central differences, one-sided on the frame border.
__global__ void k_grey_grad(const float *__restrict__ I, int W, int H, int T, float *__restrict__ gx,
                            float *__restrict__ gy)
{
    const long long n = (long long)W * H * T;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int t = (int)(i / ((long long)W * H));
        const int r = (int)(i - (long long)t * W * H);
        const int y = r / W, x = r - y * W;
        const float *f = I + (long long)t * W * H;
        float a = 0.0f, b = 0.0f;
        if (W > 1)
            a = x == 0 ? f[r + 1] - f[r] : (x == W - 1 ? f[r] - f[r - 1] : (f[r + 1] - f[r - 1]) / 2.0f);
        if (H > 1)
            b = y == 0 ? f[r + W] - f[r] : (y == H - 1 ? f[r] - f[r - W] : (f[r + W] - f[r - W]) / 2.0f);
        gx[i] = a;
        gy[i] = b;
    }
}

// One IRLS Gauss-Newton accumulation for frame pairs (n, n+1), n = blockIdx.y,
// at one level: per block the 29 sums of its PIX_PER_THREAD * 256 pixels.
__global__ void __launch_bounds__(256) k_affine_normal(const float *__restrict__ I, const uint8_t *__restrict__ occ,
                                                       const float *__restrict__ gx, const float *__restrict__ gy,
                                                       int W, int H, const double *__restrict__ mats,
                                                       const double *__restrict__ cvals, double *__restrict__ part)
{
    const int n = blockIdx.y;
    const long long HW = (long long)W * H;
    const float *I1 = I + n * HW, *I2 = I + (n + 1) * HW;
    const uint8_t *o1 = occ + n * HW, *o2 = occ + (n + 1) * HW;
    const float *gx2 = gx + (n + 1) * HW, *gy2 = gy + (n + 1) * HW;
    double m[6];
#pragma unroll
    for (int j = 0; j < 6; ++j)
        m[j] = mats[6 * n + j];
    const double cd = cvals[n];
    const bool ls = !(cd < 1e300);          // plain least squares
    const float c = (float)cd;
    float acc[NRED];
#pragma unroll
    for (int j = 0; j < NRED; ++j)
        acc[j] = 0.0f;
    const long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * PIX_PER_THREAD;
    for (int k = 0; k < PIX_PER_THREAD; ++k) {
        const long long p = base + k;
        if (p >= HW || o1[p])
            continue;
        const int y = (int)(p / W), x = (int)(p - (long long)y * W);
        double qx, qy;
        affine_apply(m, (double)x, (double)y, qx, qy);
        if (!(qx >= 0.0 && qx <= (double)(W - 1) && qy >= 0.0 && qy <= (double)(H - 1)))
            continue;
        const Tap t = make_tap(qx, qy, W, H);
        if (tap_touches(o2, t))
            continue;
        const float r = tap_value(I2, t) - I1[p];
        float w = 1.0f;
        if (!ls) {
            if (fabsf(r) < c) {
                const float u = r / c;
                w = (1.0f - u * u) * (1.0f - u * u);
            } else {
                w = 0.0f;
            }
        }
        if (w == 0.0f)
            continue;
        const float ga = tap_value(gx2, t), gb = tap_value(gy2, t);
        const float fx = (float)x, fy = (float)y;
        const float J[6] = {ga, ga * fx, ga * fy, gb, gb * fx, gb * fy};
        int idx = 0;
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int j = i; j < 6; ++j)
                acc[idx++] += w * J[i] * J[j];
#pragma unroll
        for (int i = 0; i < 6; ++i)
            acc[21 + i] += w * J[i] * r;
        acc[27] += w * r * r;
        acc[28] += w;
    }
    // block sum in FP64, fixed order: warp shuffles, then the warps in order
    __shared__ double sh[8][NRED];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NRED; ++j) {
        double v = (double)acc[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0)
            sh[warp][j] = v;
    }
    __syncthreads();
    if (threadIdx.x < NRED) {
        double s = 0.0;
        for (int wv = 0; wv < 8; ++wv)
            s += sh[wv][threadIdx.x];
        part[((long long)n * gridDim.x + blockIdx.x) * NRED + threadIdx.x] = s;
    }
}

// The block sums of every pair, in block order: out[n][29].
__global__ void k_affine_reduce(const double *__restrict__ part, int nblk, double *__restrict__ out)
{
    const int n = blockIdx.x;
    if (threadIdx.x < NRED) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b)
            s += part[((long long)n * nblk + b) * NRED + threadIdx.x];
        out[n * NRED + threadIdx.x] = s;
    }
}

// AlignVideo: frame n sampled at A_n^-1(q) (mats holds the inverses).
__global__ void k_affine_align(const float *__restrict__ rgb, const uint8_t *__restrict__ mask, int W, int H,
                               int T, const double *__restrict__ inv, float *__restrict__ out,
                               uint8_t *__restrict__ mout)
{
    const long long HW = (long long)W * H, n_all = HW * T;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_all;
         i += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(i / HW);
        const long long r = i - n * HW;
        const int y = (int)(r / W), x = (int)(r - (long long)y * W);
        double px, py;
        affine_apply(inv + 6 * n, (double)x, (double)y, px, py);
        const bool inside = px >= 0.0 && px <= (double)(W - 1) && py >= 0.0 && py <= (double)(H - 1);
        float v0 = 0.0f, v1 = 0.0f, v2 = 0.0f;
        uint8_t oc = 1;
        if (inside) {
            const Tap t = make_tap(px, py, W, H);
            const float *f = rgb + 3 * n * HW;
            v0 = tap_value(f, t, 3, 0);
            v1 = tap_value(f, t, 3, 1);
            v2 = tap_value(f, t, 3, 2);
            oc = tap_touches(mask + n * HW, t) ? 1 : 0;
        }
        out[3 * i] = v0;
        out[3 * i + 1] = v1;
        out[3 * i + 2] = v2;
        mout[i] = oc;
    }
}

// UnwarpVideo: occluded pixels y of frame n take the aligned result at A_n(y)
// (clamped to the frame); the others keep the input.
__global__ void k_affine_unwarp(const float *__restrict__ rgb, const uint8_t *__restrict__ mask,
                                const float *__restrict__ res, int W, int H, int T,
                                const double *__restrict__ fwd, float *__restrict__ out)
{
    const long long HW = (long long)W * H, n_all = HW * T;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_all;
         i += (long long)gridDim.x * blockDim.x) {
        if (!mask[i]) {
            out[3 * i] = rgb[3 * i];
            out[3 * i + 1] = rgb[3 * i + 1];
            out[3 * i + 2] = rgb[3 * i + 2];
            continue;
        }
        const int n = (int)(i / HW);
        const long long r = i - n * HW;
        const int y = (int)(r / W), x = (int)(r - (long long)y * W);
        double qx, qy;
        affine_apply(fwd + 6 * n, (double)x, (double)y, qx, qy);
        qx = fmin(fmax(qx, 0.0), (double)(W - 1));
        qy = fmin(fmax(qy, 0.0), (double)(H - 1));
        const Tap t = make_tap(qx, qy, W, H);
        const float *f = res + 3 * n * HW;
        out[3 * i] = tap_value(f, t, 3, 0);
        out[3 * i + 1] = tap_value(f, t, 3, 1);
        out[3 * i + 2] = tap_value(f, t, 3, 2);
    }
}

int grid_for(long long n)
{
    long long g = (n + 255) / 256;
    return (int)std::max(1ll, std::min(g, 152ll * 32));
}

// Solves (A + ridge I) x = -b for the 6x6 symmetric A (upper triangle packed
// row by row, as accumulated) by Gaussian elimination with partial pivoting
// in double. Returns false when singular.
bool solve6(const double *s, double *x)
{
    double A[6][7];
    int idx = 0;
    for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j) {
            A[i][j] = s[idx];
            A[j][i] = s[idx];
            ++idx;
        }
    double tr = 0.0;
    for (int i = 0; i < 6; ++i)
        tr += A[i][i];
    const double ridge = 1e-9 * (tr / 6.0) + 1e-30;
    for (int i = 0; i < 6; ++i) {
        A[i][i] += ridge;
        A[i][6] = -s[21 + i];
    }
    for (int c = 0; c < 6; ++c) {
        int piv = c;
        for (int r = c + 1; r < 6; ++r)
            if (std::fabs(A[r][c]) > std::fabs(A[piv][c]))
                piv = r;
        if (!(std::fabs(A[piv][c]) > 0.0))
            return false;
        if (piv != c)
            for (int k = 0; k < 7; ++k)
                std::swap(A[c][k], A[piv][k]);
        for (int r = c + 1; r < 6; ++r) {
            const double f = A[r][c] / A[c][c];
            for (int k = c; k < 7; ++k)
                A[r][k] -= f * A[c][k];
        }
    }
    for (int i = 5; i >= 0; --i) {
        double v = A[i][6];
        for (int k = i + 1; k < 6; ++k)
            v -= A[i][k] * x[k];
        x[i] = v / A[i][i];
    }
    for (int i = 0; i < 6; ++i)
        if (!std::isfinite(x[i]))
            return false;
    return true;
}

struct DevBuf {
    void *p = nullptr;
    cudaStream_t st = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf()
    {
        if (p)
            cudaFreeAsync(p, st);
    }
};

template <typename P>
vi_status dev_alloc(DevBuf &b, P **ptr, size_t bytes, cudaStream_t st)
{
    b.st = st;
    cudaError_t e = cudaMallocAsync(&b.p, bytes ? bytes : 16, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return rfail(e == cudaErrorMemoryAllocation ? VI_ERR_OOM : VI_ERR_CUDA, "vi_affine: allocation failed");
    }
    *ptr = (P *)b.p;
    return VI_OK;
}

#define RTRY(expr)                                                                                \
    do {                                                                                          \
        vi_status s_ = (expr);                                                                    \
        if (s_ != VI_OK)                                                                          \
            return s_;                                                                            \
    } while (0)

// Device copies of the inputs when they are host pointers.
vi_status inputs_on_device(const float *rgb, const uint8_t *mask, size_t V, int ptr_is_device, cudaStream_t st,
                           DevBuf &brgb, DevBuf &bmask, const float **drgb, const uint8_t **dmask)
{
    if (ptr_is_device) {
        *drgb = rgb;
        *dmask = mask;
        return VI_OK;
    }
    float *r = nullptr;
    uint8_t *m = nullptr;
    RTRY(dev_alloc(brgb, &r, V * 3 * sizeof(float), st));
    RTRY(dev_alloc(bmask, &m, V, st));
    RCK(cudaMemcpyAsync(r, rgb, V * 3 * sizeof(float), cudaMemcpyHostToDevice, st));
    RCK(cudaMemcpyAsync(m, mask, V, cudaMemcpyHostToDevice, st));
    *drgb = r;
    *dmask = m;
    return VI_OK;
}

bool sizes_ok(int W, int H, int T) { return W > 0 && H > 0 && T > 0 && (long long)W * H * T < (1ll << 31); }

}  // namespace
}  // namespace vi

using namespace vi;

extern "C" {

const char *vi_realign_last_error(void) { return g_realign_err.c_str(); }

int vi_affine_levels(int W, int H)
{
    int L = 1;
    while (L < 6 && (std::min(W, H) + (1 << L) - 1) / (1 << L) >= 16)
        ++L;
    return L;
}

static vi_status vi_affine_estimate_body(const float *rgb, const uint8_t *mask, int W, int H, int T, int ptr_is_device,
                             int levels, int iters, double *theta_out, void *cuda_stream)
{
    if (!rgb || !mask || !theta_out || !sizes_ok(W, H, T) || iters < 0 || iters > 1000 || levels < 0 ||
        levels > 12)
        return rfail(VI_ERR_ARG, "vi_affine_estimate: bad argument");
    const int P = T - 1;
    if (P == 0)
        return VI_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t V = (size_t)W * H * T;
    if (levels == 0)
        levels = vi_affine_levels(W, H);
    DevBuf brgb, bmask;
    const float *drgb;
    const uint8_t *dmask;
    RTRY(inputs_on_device(rgb, mask, V, ptr_is_device, st, brgb, bmask, &drgb, &dmask));

    // pyramid: grey, occlusion, gradients per level (finest first)
    std::vector<int> Ws(levels), Hs(levels);
    std::vector<DevBuf> bI(levels), bO(levels), bGx(levels), bGy(levels);
    std::vector<float *> dI(levels), dGx(levels), dGy(levels);
    std::vector<uint8_t *> dO(levels);
    Ws[0] = W;
    Hs[0] = H;
    for (int l = 1; l < levels; ++l) {
        Ws[l] = (Ws[l - 1] + 1) / 2;
        Hs[l] = (Hs[l - 1] + 1) / 2;
    }
    for (int l = 0; l < levels; ++l) {
        const size_t n = (size_t)Ws[l] * Hs[l] * T;
        RTRY(dev_alloc(bI[l], &dI[l], n * sizeof(float), st));
        RTRY(dev_alloc(bO[l], &dO[l], n, st));
        RTRY(dev_alloc(bGx[l], &dGx[l], n * sizeof(float), st));
        RTRY(dev_alloc(bGy[l], &dGy[l], n * sizeof(float), st));
    }
    VI_COUNT_LAUNCH();
    k_grey<<<grid_for((long long)V), 256, 0, st>>>(drgb, dmask, (long long)V, dI[0], dO[0]);
    for (int l = 1; l < levels; ++l) {
        VI_COUNT_LAUNCH();
        k_grey_down<<<grid_for((long long)Ws[l] * Hs[l] * T), 256, 0, st>>>(dI[l - 1], dO[l - 1], Ws[l - 1],
                                                                            Hs[l - 1], T, dI[l], dO[l], Ws[l],
                                                                            Hs[l]);
    }
    for (int l = 0; l < levels; ++l) {
        VI_COUNT_LAUNCH();
        k_grey_grad<<<grid_for((long long)Ws[l] * Hs[l] * T), 256, 0, st>>>(dI[l], Ws[l], Hs[l], T, dGx[l],
                                                                            dGy[l]);
    }
    RCK(cudaGetLastError());

    // per pair: parameters, c, partial sums
    const int nblk0 = (int)(((long long)W * H + 256LL * PIX_PER_THREAD - 1) / (256LL * PIX_PER_THREAD));
    DevBuf bM, bC, bPart, bSum;
    double *dM, *dC, *dPart, *dSum;
    RTRY(dev_alloc(bM, &dM, sizeof(double) * 6 * P, st));
    RTRY(dev_alloc(bC, &dC, sizeof(double) * P, st));
    RTRY(dev_alloc(bPart, &dPart, sizeof(double) * NRED * (size_t)nblk0 * P, st));
    RTRY(dev_alloc(bSum, &dSum, sizeof(double) * NRED * P, st));
    std::vector<double> theta(6 * (size_t)P, 0.0), c(P, INFINITY), mats(6 * (size_t)P), sums(NRED * (size_t)P);
    for (int lev = levels - 1; lev >= 0; --lev) {
        const int w = Ws[lev], h = Hs[lev];
        const int nblk = (int)(((long long)w * h + 256LL * PIX_PER_THREAD - 1) / (256LL * PIX_PER_THREAD));
        for (int it = 0; it < iters; ++it) {
            for (int n = 0; n < P; ++n) {
                const Aff a = from_theta(&theta[6 * n]);
                std::memcpy(&mats[6 * n], a.m, sizeof(a.m));
            }
            RCK(cudaMemcpyAsync(dM, mats.data(), sizeof(double) * 6 * P, cudaMemcpyHostToDevice, st));
            RCK(cudaMemcpyAsync(dC, c.data(), sizeof(double) * P, cudaMemcpyHostToDevice, st));
            VI_COUNT_LAUNCH();
            k_affine_normal<<<dim3(nblk, P), 256, 0, st>>>(dI[lev], dO[lev], dGx[lev], dGy[lev], w, h, dM, dC,
                                                           dPart);
            VI_COUNT_LAUNCH();
            k_affine_reduce<<<P, 32, 0, st>>>(dPart, nblk, dSum);
            RCK(cudaGetLastError());
            RCK(cudaMemcpyAsync(sums.data(), dSum, sizeof(double) * NRED * P, cudaMemcpyDeviceToHost, st));
            RCK(cudaStreamSynchronize(st));
            for (int n = 0; n < P; ++n) {
                const double *s = &sums[NRED * n];
                const double swr2 = s[27], sw = s[28];
                double d[6] = {0, 0, 0, 0, 0, 0};
                if (sw > 0.0 && !solve6(s, d))
                    for (double &v : d)
                        v = 0.0;
                if (sw > 0.0) {
                    for (int j = 0; j < 6; ++j)
                        theta[6 * n + j] += d[j];
                    c[n] = TUKEY_C * std::max(std::sqrt(swr2 / sw), SIGMA_FLOOR);
                }
            }
        }
        if (lev > 0)
            for (int n = 0; n < P; ++n) {
                double *a = &theta[6 * n];
                a[0] = 2.0 * a[0] - 0.5 * (a[1] + a[2]);
                a[3] = 2.0 * a[3] - 0.5 * (a[4] + a[5]);
            }
    }
    std::memcpy(theta_out, theta.data(), sizeof(double) * 6 * P);
    return VI_OK;
}

vi_status vi_affine_estimate(const float *rgb, const uint8_t *mask, int W, int H, int T, int ptr_is_device,
                             int levels, int iters, double *theta_out, void *cuda_stream)
{
    // host allocations proportional to the clip may throw; no exception crosses the C ABI
    try {
        return vi_affine_estimate_body(rgb, mask, W, H, T, ptr_is_device, levels, iters, theta_out, cuda_stream);
    } catch (...) {
        return VI_ERR_OOM;
    }
}

static vi_status vi_affine_to_reference_body(const double *theta_pairs, int T, double *to_ref_out)
{
    if (!to_ref_out || T <= 0 || (T > 1 && !theta_pairs))
        return rfail(VI_ERR_ARG, "vi_affine_to_reference: bad argument");
    const int r = std::max(0, T / 2 - 1);
    std::vector<Aff> out(T);
    const double zero[6] = {0, 0, 0, 0, 0, 0};
    out[r] = from_theta(zero);
    for (int n = r - 1; n >= 0; --n)
        out[n] = compose(out[n + 1], from_theta(theta_pairs + 6 * n));
    for (int n = r + 1; n < T; ++n)
        out[n] = compose(out[n - 1], invert(from_theta(theta_pairs + 6 * (n - 1))));
    for (int n = 0; n < T; ++n)
        to_theta(out[n], to_ref_out + 6 * n);
    return VI_OK;
}

vi_status vi_affine_to_reference(const double *theta_pairs, int T, double *to_ref_out)
{
    // host allocations proportional to the clip may throw; no exception crosses the C ABI
    try {
        return vi_affine_to_reference_body(theta_pairs, T, to_ref_out);
    } catch (...) {
        return VI_ERR_OOM;
    }
}

static vi_status vi_affine_align_body(const float *rgb, const uint8_t *mask, int W, int H, int T, const double *to_ref,
                          float *rgb_out, uint8_t *mask_out, int ptr_is_device, void *cuda_stream)
{
    if (!rgb || !mask || !to_ref || !rgb_out || !mask_out || !sizes_ok(W, H, T))
        return rfail(VI_ERR_ARG, "vi_affine_align: bad argument");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t V = (size_t)W * H * T;
    DevBuf brgb, bmask, bout, bmo, binv;
    const float *drgb;
    const uint8_t *dmask;
    RTRY(inputs_on_device(rgb, mask, V, ptr_is_device, st, brgb, bmask, &drgb, &dmask));
    float *dout = rgb_out;
    uint8_t *dmo = mask_out;
    if (!ptr_is_device) {
        RTRY(dev_alloc(bout, &dout, V * 3 * sizeof(float), st));
        RTRY(dev_alloc(bmo, &dmo, V, st));
    }
    std::vector<double> inv(6 * (size_t)T);
    for (int n = 0; n < T; ++n) {
        const Aff a = invert(from_theta(to_ref + 6 * n));
        std::memcpy(&inv[6 * n], a.m, sizeof(a.m));
    }
    double *dinv;
    RTRY(dev_alloc(binv, &dinv, sizeof(double) * 6 * T, st));
    RCK(cudaMemcpyAsync(dinv, inv.data(), sizeof(double) * 6 * T, cudaMemcpyHostToDevice, st));
    VI_COUNT_LAUNCH();
    k_affine_align<<<grid_for((long long)V), 256, 0, st>>>(drgb, dmask, W, H, T, dinv, dout, dmo);
    RCK(cudaGetLastError());
    if (!ptr_is_device) {
        RCK(cudaMemcpyAsync(rgb_out, dout, V * 3 * sizeof(float), cudaMemcpyDeviceToHost, st));
        RCK(cudaMemcpyAsync(mask_out, dmo, V, cudaMemcpyDeviceToHost, st));
    }
    RCK(cudaStreamSynchronize(st));
    return VI_OK;
}

vi_status vi_affine_align(const float *rgb, const uint8_t *mask, int W, int H, int T, const double *to_ref,
                          float *rgb_out, uint8_t *mask_out, int ptr_is_device, void *cuda_stream)
{
    // host allocations proportional to the clip may throw; no exception crosses the C ABI
    try {
        return vi_affine_align_body(rgb, mask, W, H, T, to_ref, rgb_out, mask_out, ptr_is_device, cuda_stream);
    } catch (...) {
        return VI_ERR_OOM;
    }
}

static vi_status vi_affine_unwarp_body(const float *rgb, const uint8_t *mask, const float *aligned_result, int W, int H,
                           int T, const double *to_ref, float *rgb_out, int ptr_is_device, void *cuda_stream)
{
    if (!rgb || !mask || !aligned_result || !to_ref || !rgb_out || !sizes_ok(W, H, T))
        return rfail(VI_ERR_ARG, "vi_affine_unwarp: bad argument");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t V = (size_t)W * H * T;
    DevBuf brgb, bmask, bres, bout, bfwd;
    const float *drgb;
    const uint8_t *dmask;
    RTRY(inputs_on_device(rgb, mask, V, ptr_is_device, st, brgb, bmask, &drgb, &dmask));
    const float *dres = aligned_result;
    float *dout = rgb_out;
    if (!ptr_is_device) {
        float *r;
        RTRY(dev_alloc(bres, &r, V * 3 * sizeof(float), st));
        RCK(cudaMemcpyAsync(r, aligned_result, V * 3 * sizeof(float), cudaMemcpyHostToDevice, st));
        dres = r;
        RTRY(dev_alloc(bout, &dout, V * 3 * sizeof(float), st));
    }
    std::vector<double> fwd(6 * (size_t)T);
    for (int n = 0; n < T; ++n) {
        const Aff a = from_theta(to_ref + 6 * n);
        std::memcpy(&fwd[6 * n], a.m, sizeof(a.m));
    }
    double *dfwd;
    RTRY(dev_alloc(bfwd, &dfwd, sizeof(double) * 6 * T, st));
    RCK(cudaMemcpyAsync(dfwd, fwd.data(), sizeof(double) * 6 * T, cudaMemcpyHostToDevice, st));
    VI_COUNT_LAUNCH();
    k_affine_unwarp<<<grid_for((long long)V), 256, 0, st>>>(drgb, dmask, dres, W, H, T, dfwd, dout);
    RCK(cudaGetLastError());
    if (!ptr_is_device)
        RCK(cudaMemcpyAsync(rgb_out, dout, V * 3 * sizeof(float), cudaMemcpyDeviceToHost, st));
    RCK(cudaStreamSynchronize(st));
    return VI_OK;
}

vi_status vi_affine_unwarp(const float *rgb, const uint8_t *mask, const float *aligned_result, int W, int H,
                           int T, const double *to_ref, float *rgb_out, int ptr_is_device, void *cuda_stream)
{
    // host allocations proportional to the clip may throw; no exception crosses the C ABI
    try {
        return vi_affine_unwarp_body(rgb, mask, aligned_result, W, H, T, to_ref, rgb_out, ptr_is_device, cuda_stream);
    } catch (...) {
        return VI_ERR_OOM;
    }
}

}  // extern "C"
