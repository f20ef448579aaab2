/*
 * vi_oracle.c -- plain, slow CPU oracle for the method of Newson, Almansa,
 * Fradet, Gousseau and Perez, "Video Inpainting of Complex Scenes"
 * (SIAM J. Imaging Sciences, 2014; arXiv:1503.05528).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the package's smoke() entry and the
 * CPU-baseline leg of the benchmark may load this library. The product path
 * (the CUDA library) shares no code, header, table or helper with it.
 *
 * Every function follows one passage of the paper, written as loops a reader
 * can check against it by eye: no blocking, fusion or reordering. Decisions
 * that turn floating point into an integer (which candidate wins, which
 * neighbour is the argmin) are taken in FP32, the precision the CUDA kernels
 * decide in; sums that only produce values (vote, features, pyramid, energy)
 * are carried in FP64.
 *
 * Layout: a level is W x H x T voxels, voxel index v = (t*H + y)*W + x
 * ("lexicographic" order, x fastest); channel c of voxel v is x[v*C + c].
 * Masks are one byte per voxel (0 or 1). A shift map phi holds (dx, dy, dt)
 * int32 triples per voxel. Patches are 5x5x5 (Sec. 3.7), offsets -2..2.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no contraction of a*b+c:
 * the FP32 distance uses fmaf explicitly and nothing else may fuse).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define R 2                 /* patch half-size: 5x5x5 patches (Sec. 3.7) */
#define NPATCH 125          /* N in Eq. 2 */

static size_t vidx(int x, int y, int t, int W, int H)
{
    return ((size_t)t * (size_t)H + (size_t)y) * (size_t)W + (size_t)x;
}

static int inside(int x, int y, int t, int W, int H, int T)
{
    return x >= 0 && x < W && y >= 0 && y < H && t >= 0 && t < T;
}

static void coords(size_t v, int W, int H, int *x, int *y, int *t)
{
    *x = (int)(v % (size_t)W);
    *y = (int)((v / (size_t)W) % (size_t)H);
    *t = (int)(v / ((size_t)W * (size_t)H));
}

/* ------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11). Ten rounds; each round multiplies words 0 and 2
 * by the two Philox constants, mixes the high halves with words 1 and 3 and
 * the round key, and the key is bumped by the two Weyl constants between
 * rounds. Written from the paper's definition.
 * ---------------------------------------------------------------------- */
void vio_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter layout shared by every random draw of the method: word 0 is the
 * voxel index at the level, word 1 a tag naming the draw, word 2 the clip. */
static void draw(uint32_t voxel, uint32_t tag, uint32_t clip, uint32_t key0, uint32_t key1,
                 uint32_t out[4])
{
    uint32_t ctr[4] = {voxel, tag, clip, 0u};
    uint32_t key[2] = {key0, key1};
    vio_philox4x32_10(ctr, key, out);
}

/* A 32-bit word read as a uniform value in (-1, 1): its 24 high bits, centred
 * in their cell: delta = ((w >> 8) + 1/2) / 2^23 - 1. */
double vio_unit_symmetric(uint32_t w)
{
    return ((double)(w >> 8) + 0.5) / 8388608.0 - 1.0;
}

/* A 32-bit word read as a uniform index in [0, n): floor(w * n / 2^32). */
uint32_t vio_uniform_index(uint32_t w, uint32_t n)
{
    return (uint32_t)(((uint64_t)w * (uint64_t)n) >> 32);
}

/* ------------------------------------------------------------------------
 * Patch distances: Eq. 2 (colour), Eq. 7b (colour + lambda-weighted texture,
 * with the texture channels stored pre-multiplied by sqrt(lambda)) and the
 * partial distance Eq. 11 of the initialisation (voxels of the current
 * occlusion H' left out, normalised by |N'_p|).
 *
 * The patch of p is the 5x5x5 cuboid of offsets (dx, dy, dt) in [-2, 2]^3,
 * taken in the predefined order dt, then dy, then dx ascending (Sec. 2: "the
 * N pixels in N_p ... are ordered in a predefined way"). Offsets whose target
 * voxel p + o lies outside the video contribute nothing; the source patch is
 * always inside (sources are in D~). Eq. 2 divides by N = 125.
 * ---------------------------------------------------------------------- */

/* FP32, summed in a fixed order (Eq. 2 itself fixes none): the terms (a - b)^2
 * of one row (fixed dt, dy; dx ascending, channels ascending) are added with
 * one fused multiply-add each, starting from 0; the 5 row sums of a slice
 * (fixed dt) are added in dy order; the 5 slice sums are added in dt order;
 * the total is divided by N (or |N'_p|). Skipped voxels add nothing. */
float vio_dist_f32(const float *x, int W, int H, int T, int C,
                   int px, int py, int pt, int sx, int sy, int st, const uint8_t *excl)
{
    if (sx - R < 0 || sy - R < 0 || st - R < 0 || sx + R >= W || sy + R >= H || st + R >= T)
        return INFINITY;
    float total = 0.0f;
    int n = 0;
    for (int dt = -R; dt <= R; ++dt) {
        float slice = 0.0f;
        for (int dy = -R; dy <= R; ++dy) {
            float row = 0.0f;
            for (int dx = -R; dx <= R; ++dx) {
                int rx = px + dx, ry = py + dy, rt = pt + dt;
                if (!inside(rx, ry, rt, W, H, T))
                    continue;
                size_t r = vidx(rx, ry, rt, W, H);
                if (excl && excl[r])
                    continue;
                size_t s = vidx(sx + dx, sy + dy, st + dt, W, H);
                for (int c = 0; c < C; ++c) {
                    float df = x[r * (size_t)C + c] - x[s * (size_t)C + c];
                    row = fmaf(df, df, row);
                }
                ++n;
            }
            slice = slice + row;
        }
        total = total + slice;
    }
    if (excl) {
        if (n == 0)
            return INFINITY;
        return total / (float)n;
    }
    return total / (float)NPATCH;
}

/* FP64 evaluation of the same definition (plain summation), for the energy
 * evaluator and for error statements against FP32. */
double vio_dist_f64(const float *x, int W, int H, int T, int C,
                    int px, int py, int pt, int sx, int sy, int st, const uint8_t *excl)
{
    if (sx - R < 0 || sy - R < 0 || st - R < 0 || sx + R >= W || sy + R >= H || st + R >= T)
        return INFINITY;
    double acc = 0.0;
    int n = 0;
    for (int dt = -R; dt <= R; ++dt)
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
                int rx = px + dx, ry = py + dy, rt = pt + dt;
                if (!inside(rx, ry, rt, W, H, T))
                    continue;
                size_t r = vidx(rx, ry, rt, W, H);
                if (excl && excl[r])
                    continue;
                size_t s = vidx(sx + dx, sy + dy, st + dt, W, H);
                for (int c = 0; c < C; ++c) {
                    double df = (double)x[r * (size_t)C + c] - (double)x[s * (size_t)C + c];
                    acc += df * df;
                }
                ++n;
            }
    if (excl) {
        if (n == 0)
            return INFINITY;
        return acc / (double)n;
    }
    return acc / (double)NPATCH;
}

/* ------------------------------------------------------------------------
 * Sets of Sec. 2: D~ = {p in D : N_p in D} (here also N_p inside the video,
 * so that every source patch is whole), and H~ = union of N_p over p in H
 * (the dilated occlusion, clipped to the video).
 * ---------------------------------------------------------------------- */
void vio_dilate5(const uint8_t *in, int W, int H, int T, uint8_t *out)
{
    for (int t = 0; t < T; ++t)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                int any = 0;
                for (int dt = -R; dt <= R && !any; ++dt)
                    for (int dy = -R; dy <= R && !any; ++dy)
                        for (int dx = -R; dx <= R && !any; ++dx) {
                            int qx = x + dx, qy = y + dy, qt = t + dt;
                            if (inside(qx, qy, qt, W, H, T) && in[vidx(qx, qy, qt, W, H)])
                                any = 1;
                        }
                out[vidx(x, y, t, W, H)] = (uint8_t)any;
            }
}

void vio_masks(const uint8_t *hole, int W, int H, int T, uint8_t *htilde, uint8_t *dtilde)
{
    vio_dilate5(hole, W, H, T, htilde);
    for (int t = 0; t < T; ++t)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                int ok = 1;
                for (int dt = -R; dt <= R && ok; ++dt)
                    for (int dy = -R; dy <= R && ok; ++dy)
                        for (int dx = -R; dx <= R && ok; ++dx) {
                            int qx = x + dx, qy = y + dy, qt = t + dt;
                            if (!inside(qx, qy, qt, W, H, T) || hole[vidx(qx, qy, qt, W, H)])
                                ok = 0;
                        }
                dtilde[vidx(x, y, t, W, H)] = (uint8_t)ok;
            }
}

/* Erosion by the 3x3x3 structuring element of Algorithm 3: p stays iff p and
 * its 26 neighbours are all in the set (voxels outside the video are not). */
void vio_erode3(const uint8_t *in, int W, int H, int T, uint8_t *out)
{
    for (int t = 0; t < T; ++t)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                int all = in[vidx(x, y, t, W, H)] ? 1 : 0;
                for (int dt = -1; dt <= 1 && all; ++dt)
                    for (int dy = -1; dy <= 1 && all; ++dy)
                        for (int dx = -1; dx <= 1 && all; ++dx) {
                            int qx = x + dx, qy = y + dy, qt = t + dt;
                            if (!inside(qx, qy, qt, W, H, T) || !in[vidx(qx, qy, qt, W, H)])
                                all = 0;
                        }
                out[vidx(x, y, t, W, H)] = (uint8_t)all;
            }
}

/* ------------------------------------------------------------------------
 * Texture features, Eq. 7: T(p) = mean over q in nu(p) of (|I_x(q)|, |I_y(q)|),
 * I the grey level (R+G+B)/3, I_x and I_y central differences (one-sided on
 * the frame border). nu(p) is the square of side s around p covering offsets
 * [-floor(s/2), -floor(s/2) + s - 1] (s = 2^(L-1), Sec. 3.3). A derivative
 * sample whose stencil reads an occluded voxel is unknown and left out of the
 * mean; with no known sample the feature is 0. Output [V][2] in FP64.
 * ---------------------------------------------------------------------- */
void vio_texture_features(const float *rgb, const uint8_t *hole, int W, int H, int T,
                          int nu_side, double *Tout)
{
    size_t F = (size_t)W * (size_t)H;
    double *I = (double *)malloc(F * sizeof(double));
    double *gx = (double *)malloc(F * sizeof(double));
    double *gy = (double *)malloc(F * sizeof(double));
    uint8_t *okx = (uint8_t *)malloc(F);
    uint8_t *oky = (uint8_t *)malloc(F);
    int lo = -(nu_side / 2), hi = lo + nu_side - 1;
    for (int t = 0; t < T; ++t) {
        const float *fr = rgb + (size_t)t * F * 3;
        const uint8_t *hm = hole + (size_t)t * F;
        for (size_t i = 0; i < F; ++i)
            I[i] = ((double)fr[3 * i] + (double)fr[3 * i + 1] + (double)fr[3 * i + 2]) / 3.0;
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                size_t i = (size_t)y * W + x;
                int a, b;
                double den;
                /* d/dx */
                if (W < 2) {
                    okx[i] = 0; gx[i] = 0.0;
                } else {
                    if (x == 0) { a = 0; b = 1; den = 1.0; }
                    else if (x == W - 1) { a = W - 2; b = W - 1; den = 1.0; }
                    else { a = x - 1; b = x + 1; den = 2.0; }
                    size_t ia = (size_t)y * W + a, ib = (size_t)y * W + b;
                    okx[i] = (uint8_t)(!hm[ia] && !hm[ib]);
                    gx[i] = (I[ib] - I[ia]) / den;
                }
                /* d/dy */
                if (H < 2) {
                    oky[i] = 0; gy[i] = 0.0;
                } else {
                    if (y == 0) { a = 0; b = 1; den = 1.0; }
                    else if (y == H - 1) { a = H - 2; b = H - 1; den = 1.0; }
                    else { a = y - 1; b = y + 1; den = 2.0; }
                    size_t ia = (size_t)a * W + x, ib = (size_t)b * W + x;
                    oky[i] = (uint8_t)(!hm[ia] && !hm[ib]);
                    gy[i] = (I[ib] - I[ia]) / den;
                }
            }
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                double sx = 0.0, sy = 0.0;
                int nx = 0, ny = 0;
                for (int j = lo; j <= hi; ++j)
                    for (int i2 = lo; i2 <= hi; ++i2) {
                        int qx = x + i2, qy = y + j;
                        if (qx < 0 || qx >= W || qy < 0 || qy >= H)
                            continue;
                        size_t q = (size_t)qy * W + qx;
                        if (okx[q]) { sx += fabs(gx[q]); ++nx; }
                        if (oky[q]) { sy += fabs(gy[q]); ++ny; }
                    }
                size_t o = ((size_t)t * F + (size_t)y * W + x) * 2;
                Tout[o] = nx ? sx / nx : 0.0;
                Tout[o + 1] = ny ? sy / ny : 0.0;
            }
    }
    free(I); free(gx); free(gy); free(okx); free(oky);
}

/* Texture pyramid, Eq. 8: T^l(x, y, t) = T(2^l x, 2^l y, t), no filtering. */
/* Eq. 8 with the temporal subsampling option: T^l(x, y, t) = T(2^l x, 2^l y,
 * t), or T(2^l x, 2^l y, 2^l t) when tsub (Tl frames at level l). */
void vio_subsample_features_t(const double *T0, int W0, int H0, int T, int level,
                              int Wl, int Hl, int Tl, int tsub, double *out)
{
    (void)T;
    for (int t = 0; t < Tl; ++t)
        for (int y = 0; y < Hl; ++y)
            for (int x = 0; x < Wl; ++x) {
                size_t src = vidx(x << level, y << level, tsub ? (t << level) : t, W0, H0);
                size_t dst = vidx(x, y, t, Wl, Hl);
                out[2 * dst] = T0[2 * src];
                out[2 * dst + 1] = T0[2 * src + 1];
            }
}

void vio_subsample_features(const double *T0, int W0, int H0, int T, int level,
                            int Wl, int Hl, double *Tl)
{
    vio_subsample_features_t(T0, W0, H0, T, level, Wl, Hl, T, 0, Tl);
}

/* Colour and occlusion pyramids (Algorithm 4, "ImagePyramid" and
 * "OcclusionPyramid"). A coarse voxel is occluded when any of its children
 * is; a known coarse voxel is the mean of its children. Children: the (up
 * to) 2x2 spatial ones of the same frame (Sec. 3.6: no temporal
 * subsampling), or with tsub the (up to) 2x2x2 of frames 2t and 2t+1 (the
 * option the paper uses once, for long occlusions). Coarse size ceil(W/2) x
 * ceil(H/2) x (tsub ? ceil(T/2) : T). */
void vio_downsample_t(const float *xf, const uint8_t *hole_f, int Wf, int Hf, int Tf, int C, int tsub,
                      float *xc, uint8_t *hole_c)
{
    int Wc = (Wf + 1) / 2, Hc = (Hf + 1) / 2, Tc = tsub ? (Tf + 1) / 2 : Tf;
    for (int t = 0; t < Tc; ++t)
        for (int y = 0; y < Hc; ++y)
            for (int x = 0; x < Wc; ++x) {
                size_t o = vidx(x, y, t, Wc, Hc);
                int occl = 0, n = 0;
                double acc[8] = {0};
                for (int k = 0; k <= (tsub ? 1 : 0); ++k)
                    for (int j = 0; j < 2; ++j)
                        for (int i = 0; i < 2; ++i) {
                            int fx = 2 * x + i, fy = 2 * y + j, ft = tsub ? 2 * t + k : t;
                            if (fx >= Wf || fy >= Hf || ft >= Tf)
                                continue;
                            size_t f = vidx(fx, fy, ft, Wf, Hf);
                            if (hole_f[f])
                                occl = 1;
                            for (int c = 0; c < C && c < 8; ++c)
                                acc[c] += (double)xf[f * (size_t)C + c];
                            ++n;
                        }
                hole_c[o] = (uint8_t)occl;
                for (int c = 0; c < C; ++c)
                    xc[o * (size_t)C + c] = occl ? 0.0f : (float)(acc[c] / n);
            }
}

void vio_downsample(const float *xf, const uint8_t *hole_f, int Wf, int Hf, int T, int C,
                    float *xc, uint8_t *hole_c)
{
    vio_downsample_t(xf, hole_f, Wf, Hf, T, C, 0, xc, hole_c);
}

/* ------------------------------------------------------------------------
 * Shift-map initialisation (Sec. 3.1, Algorithm 4 "phi^L <- Random"): each
 * target takes a uniformly drawn source of D~ (raster-ordered list).
 * ---------------------------------------------------------------------- */
static size_t *source_list(const uint8_t *dtilde, size_t V, size_t *n)
{
    size_t cnt = 0;
    for (size_t v = 0; v < V; ++v)
        cnt += dtilde[v] ? 1 : 0;
    size_t *list = (size_t *)malloc((cnt ? cnt : 1) * sizeof(size_t));
    size_t k = 0;
    for (size_t v = 0; v < V; ++v)
        if (dtilde[v])
            list[k++] = v;
    *n = cnt;
    return list;
}

int vio_init_nnf(const uint8_t *target, const uint8_t *dtilde, int W, int H, int T,
                 uint32_t key0, uint32_t key1, uint32_t tag, uint32_t clip, int32_t *phi)
{
    size_t V = (size_t)W * H * T, nS;
    size_t *src = source_list(dtilde, V, &nS);
    if (nS == 0) { free(src); return -1; }
    for (size_t p = 0; p < V; ++p) {
        if (!target[p])
            continue;
        uint32_t w[4];
        draw((uint32_t)p, tag, clip, key0, key1, w);
        size_t s = src[vio_uniform_index(w[0], (uint32_t)nS)];
        int px, py, pt, sx, sy, st;
        coords(p, W, H, &px, &py, &pt);
        coords(s, W, H, &sx, &sy, &st);
        phi[3 * p] = sx - px; phi[3 * p + 1] = sy - py; phi[3 * p + 2] = st - pt;
    }
    free(src);
    return 0;
}

/* Level transition (Sec. 3.6, Algorithm 4 "UpSample(phi, 2)"): the fine voxel
 * (x, y, t) takes the shift of its coarse parent (x/2, y/2, t) with the spatial
 * components doubled (nearest-neighbour upsampling; no temporal scaling), or,
 * with the temporal subsampling option (tsub), of the parent (x/2, y/2, t/2)
 * with all three components doubled. A shift that does not land in the fine
 * D~ is redrawn uniformly from D~. */
int vio_upsample_nnf_t(const int32_t *phi_c, int Wc, int Hc, int Tc, const uint8_t *target_f,
                       const uint8_t *dtilde_f, int Wf, int Hf, int Tf, int tsub,
                       uint32_t key0, uint32_t key1, uint32_t tag, uint32_t clip, int32_t *phi_f)
{
    (void)Tc;
    size_t V = (size_t)Wf * Hf * Tf, nS;
    size_t *src = source_list(dtilde_f, V, &nS);
    if (nS == 0) { free(src); return -1; }
    for (size_t p = 0; p < V; ++p) {
        if (!target_f[p])
            continue;
        int px, py, pt;
        coords(p, Wf, Hf, &px, &py, &pt);
        size_t P = vidx(px / 2, py / 2, tsub ? pt / 2 : pt, Wc, Hc);
        int dx = 2 * phi_c[3 * P], dy = 2 * phi_c[3 * P + 1], dt = (tsub ? 2 : 1) * phi_c[3 * P + 2];
        int sx = px + dx, sy = py + dy, st = pt + dt;
        if (!(inside(sx, sy, st, Wf, Hf, Tf) && dtilde_f[vidx(sx, sy, st, Wf, Hf)])) {
            uint32_t w[4];
            draw((uint32_t)p, tag, clip, key0, key1, w);
            size_t s = src[vio_uniform_index(w[0], (uint32_t)nS)];
            coords(s, Wf, Hf, &sx, &sy, &st);
            dx = sx - px; dy = sy - py; dt = st - pt;
        }
        phi_f[3 * p] = dx; phi_f[3 * p + 1] = dy; phi_f[3 * p + 2] = dt;
    }
    free(src);
    return 0;
}

int vio_upsample_nnf(const int32_t *phi_c, int Wc, int Hc, const uint8_t *target_f,
                     const uint8_t *dtilde_f, int Wf, int Hf, int T,
                     uint32_t key0, uint32_t key1, uint32_t tag, uint32_t clip, int32_t *phi_f)
{
    return vio_upsample_nnf_t(phi_c, Wc, Hc, T, target_f, dtilde_f, Wf, Hf, T, 0, key0, key1, tag, clip,
                              phi_f);
}

/* ------------------------------------------------------------------------
 * ANN search with 3D PatchMatch (Sec. 3.1, Algorithm 1).
 *
 * Targets are the voxels with target[p] = 1 (H~ in the main loop, the
 * patches meeting the current layer during the initialisation). First the
 * distance of every target to its current correspondent is evaluated; then,
 * for k = 1..n_pm:
 *   propagation -- candidates phi(p - e_x), phi(p - e_y), phi(p - e_t) on even
 *     k, phi(p + e_x), phi(p + e_y), phi(p + e_t) on odd k, taken in that
 *     order; a candidate counts only if the neighbour is a target and
 *     p + phi(neighbour) is in D~; it replaces phi(p) only if strictly closer.
 *   random search (Eq. 3) -- candidate p + phi(p) + floor(r_max rho^k delta),
 *     delta uniform in (-1, 1)^3 from Philox (counter: voxel, tag | k, clip);
 *     accepted if it lies in D~ and is strictly closer.
 *
 * schedule 0 (SEQ) is Algorithm 1 as printed: the propagation scans targets in
 *   lexicographic order on even k and in reverse order on odd k, updating phi
 *   in place, so a shift travels along the whole scan in one sweep.
 * schedule 1 (JAC) is the parallel schedule: every target of sweep k reads its
 *   neighbours' shifts as they were when sweep k began.
 * The random search reads only phi(p), so it is the same in both.
 *
 * phi (int32 x3 per voxel) and d2 (float per voxel) are updated for targets.
 * excl != NULL selects the partial distance of Eq. 11. Returns the number of
 * distance evaluations performed.
 * ---------------------------------------------------------------------- */
typedef struct {
    const float *x; int W, H, T, C;
    const uint8_t *target, *dtilde, *excl;
    long long evals;
    int fp64;   /* 0: FP32 distances (the canonical order); 1: FP64 distances */
} ann_ctx;

/* The distance the search compares, held in double: the FP32 one converted
 * exactly (so comparisons decide as in FP32), or the FP64 one. */
static double ann_dist(const ann_ctx *a, int px, int py, int pt, int sx, int sy, int st)
{
    if (a->fp64)
        return vio_dist_f64(a->x, a->W, a->H, a->T, a->C, px, py, pt, sx, sy, st, a->excl);
    return (double)vio_dist_f32(a->x, a->W, a->H, a->T, a->C, px, py, pt, sx, sy, st, a->excl);
}

static void try_shift(ann_ctx *a, int px, int py, int pt, int cdx, int cdy, int cdt,
                      int32_t *bphi, double *bd)
{
    int sx = px + cdx, sy = py + cdy, st = pt + cdt;
    if (!inside(sx, sy, st, a->W, a->H, a->T))
        return;
    if (!a->dtilde[vidx(sx, sy, st, a->W, a->H)])
        return;
    double d = ann_dist(a, px, py, pt, sx, sy, st);
    a->evals++;
    if (d < *bd) {
        *bd = d;
        bphi[0] = cdx; bphi[1] = cdy; bphi[2] = cdt;
    }
}

static void propagate_one(ann_ctx *a, size_t p, int k, const int32_t *phi_src,
                          int32_t *phi, double *d2)
{
    int W = a->W, H = a->H, T = a->T;
    int px, py, pt;
    coords(p, W, H, &px, &py, &pt);
    int sgn = (k % 2 == 0) ? -1 : +1;
    int32_t best[3] = {phi[3 * p], phi[3 * p + 1], phi[3 * p + 2]};
    double bd = d2[p];
    int nb[3][3] = {{px + sgn, py, pt}, {px, py + sgn, pt}, {px, py, pt + sgn}};
    for (int i = 0; i < 3; ++i) {
        int rx = nb[i][0], ry = nb[i][1], rt = nb[i][2];
        if (!inside(rx, ry, rt, W, H, T))
            continue;
        size_t r = vidx(rx, ry, rt, W, H);
        if (!a->target[r])
            continue;
        try_shift(a, px, py, pt, phi_src[3 * r], phi_src[3 * r + 1], phi_src[3 * r + 2], best, &bd);
    }
    phi[3 * p] = best[0]; phi[3 * p + 1] = best[1]; phi[3 * p + 2] = best[2];
    d2[p] = bd;
}

/* The random search of iteration k around the target's current shift.
 * rs_mode 0 (Algorithm 1, Eq. 3): one candidate at radius r_max rho^k,
 * drawn from counter (p, tag | k, clip, 0). rs_mode 1 (the original
 * PatchMatch's search): candidates at every radius r_max rho^i >= 1, i = 0,
 * 1, ..., largest first, each drawn from counter (p, tag | k, clip, i) around
 * the best shift so far. */
static void random_search_one(ann_ctx *a, size_t p, int k, int rmax, double rho, int rs_mode,
                              uint32_t key0, uint32_t key1, uint32_t tag_base, uint32_t clip,
                              int32_t *phi, double *d2)
{
    int px, py, pt;
    coords(p, a->W, a->H, &px, &py, &pt);
    int32_t best[3] = {phi[3 * p], phi[3 * p + 1], phi[3 * p + 2]};
    double bd = d2[p];
    for (int i = 0;; ++i) {
        double radius;
        uint32_t w[4];
        uint32_t ctr[4] = {(uint32_t)p, tag_base | (uint32_t)k, clip, 0u};
        uint32_t key[2] = {key0, key1};
        if (rs_mode == 0) {
            radius = (double)rmax * pow(rho, (double)k);
        } else {
            radius = (double)rmax * pow(rho, (double)i);
            if (radius < 1.0)
                break;
            ctr[3] = (uint32_t)i;
        }
        vio_philox4x32_10(ctr, key, w);
        int ox = (int)floor(radius * vio_unit_symmetric(w[0]));
        int oy = (int)floor(radius * vio_unit_symmetric(w[1]));
        int ot = (int)floor(radius * vio_unit_symmetric(w[2]));
        try_shift(a, px, py, pt, best[0] + ox, best[1] + oy, best[2] + ot, best, &bd);
        if (rs_mode == 0)
            break;
    }
    phi[3 * p] = best[0]; phi[3 * p + 1] = best[1]; phi[3 * p + 2] = best[2];
    d2[p] = bd;
}

/* Algorithm 1 on the targets, in place on (phi, d2); returns the number of
 * distance evaluations (candidates that land in D~, plus the initial
 * distances). schedule 0: the sequential sweep as printed (in-place
 * propagation in scan order); 1: Jacobi (every target reads the shifts the
 * sweep started from). sub_sweeps >= 1 propagation sweeps (same direction)
 * run before the random search of each iteration k; rs_mode as in
 * random_search_one. */
static long long ann_core(const float *x, int W, int H, int T, int C,
                          const uint8_t *target, const uint8_t *dtilde, const uint8_t *excl,
                          int32_t *phi, double *d2, int n_pm, int schedule, int rmax, double rho,
                          uint32_t key0, uint32_t key1, uint32_t tag_base, uint32_t clip, int rs_mode,
                          int sub_sweeps, int fp64)
{
    size_t V = (size_t)W * H * T;
    ann_ctx a = {x, W, H, T, C, target, dtilde, excl, 0, fp64};

    /* distance of each target to its current correspondent */
    for (size_t p = 0; p < V; ++p) {
        if (!target[p])
            continue;
        int px, py, pt;
        coords(p, W, H, &px, &py, &pt);
        int sx = px + phi[3 * p], sy = py + phi[3 * p + 1], st = pt + phi[3 * p + 2];
        if (inside(sx, sy, st, W, H, T) && dtilde[vidx(sx, sy, st, W, H)]) {
            d2[p] = ann_dist(&a, px, py, pt, sx, sy, st);
            a.evals++;
        } else {
            d2[p] = INFINITY;
        }
    }

    int32_t *phi_old = NULL;
    if (schedule == 1)
        phi_old = (int32_t *)malloc(V * 3 * sizeof(int32_t));

    for (int k = 1; k <= n_pm; ++k) {
        for (int j = 0; j < sub_sweeps; ++j) {
            if (schedule == 0) {
                if (k % 2 == 0) {
                    for (size_t p = 0; p < V; ++p)
                        if (target[p])
                            propagate_one(&a, p, k, phi, phi, d2);
                } else {
                    for (size_t i = V; i-- > 0;)
                        if (target[i])
                            propagate_one(&a, i, k, phi, phi, d2);
                }
            } else {
                memcpy(phi_old, phi, V * 3 * sizeof(int32_t));
                for (size_t p = 0; p < V; ++p)
                    if (target[p])
                        propagate_one(&a, p, k, phi_old, phi, d2);
            }
        }
        for (size_t p = 0; p < V; ++p)
            if (target[p])
                random_search_one(&a, p, k, rmax, rho, rs_mode, key0, key1, tag_base, clip, phi, d2);
    }
    free(phi_old);
    return a.evals;
}

/* FP32 distances in and out as float (exact both ways). */
static double *widen(const float *d2, size_t V)
{
    double *w = (double *)malloc(V * sizeof(double));
    if (w)
        for (size_t v = 0; v < V; ++v)
            w[v] = (double)d2[v];
    return w;
}

static void narrow(const double *w, float *d2, size_t V)
{
    for (size_t v = 0; v < V; ++v)
        d2[v] = (float)w[v];
}

long long vio_ann2(const float *x, int W, int H, int T, int C,
                   const uint8_t *target, const uint8_t *dtilde, const uint8_t *excl,
                   int32_t *phi, float *d2, int n_pm, int schedule, int rmax, double rho,
                   uint32_t key0, uint32_t key1, uint32_t tag_base, uint32_t clip, int rs_mode,
                   int sub_sweeps)
{
    size_t V = (size_t)W * H * T;
    double *w = widen(d2, V);
    if (!w)
        return -1;
    long long n = ann_core(x, W, H, T, C, target, dtilde, excl, phi, w, n_pm, schedule, rmax, rho, key0, key1,
                           tag_base, clip, rs_mode, sub_sweeps, 0);
    narrow(w, d2, V);
    free(w);
    return n;
}

/* The same search with FP64 distances and decisions (d2 in double): the
 * reference the FP32 path's errors are stated against. */
long long vio_ann2_f64(const float *x, int W, int H, int T, int C,
                       const uint8_t *target, const uint8_t *dtilde, const uint8_t *excl,
                       int32_t *phi, double *d2, int n_pm, int schedule, int rmax, double rho,
                       uint32_t key0, uint32_t key1, uint32_t tag_base, uint32_t clip, int rs_mode,
                       int sub_sweeps)
{
    return ann_core(x, W, H, T, C, target, dtilde, excl, phi, d2, n_pm, schedule, rmax, rho, key0, key1,
                    tag_base, clip, rs_mode, sub_sweeps, 1);
}

/* The two parts of vio_ann2's Jacobi schedule on their own, so that ranks
 * holding different targets can exchange shifts between iterations: the
 * distance of every target to its current correspondent (+inf where that is
 * not in D~), and one iteration k (sub_sweeps Jacobi propagation sweeps, then
 * the random search) for the targets marked in own (NULL: every target),
 * where target still says which neighbours hold a shift. vio_rescore
 * followed by vio_ann_iteration for k = 1 .. n_pm is vio_ann2 with schedule
 * 1, step for step. Each returns its evaluations. */
long long vio_rescore(const float *x, int W, int H, int T, int C, const uint8_t *target,
                      const uint8_t *dtilde, const uint8_t *excl, const int32_t *phi, float *d2)
{
    size_t V = (size_t)W * H * T;
    long long evals = 0;
    for (size_t p = 0; p < V; ++p) {
        if (!target[p])
            continue;
        int px, py, pt;
        coords(p, W, H, &px, &py, &pt);
        int sx = px + phi[3 * p], sy = py + phi[3 * p + 1], st = pt + phi[3 * p + 2];
        if (inside(sx, sy, st, W, H, T) && dtilde[vidx(sx, sy, st, W, H)]) {
            d2[p] = vio_dist_f32(x, W, H, T, C, px, py, pt, sx, sy, st, excl);
            evals++;
        } else {
            d2[p] = INFINITY;
        }
    }
    return evals;
}

long long vio_ann_iteration(const float *x, int W, int H, int T, int C, const uint8_t *target,
                            const uint8_t *own, const uint8_t *dtilde, const uint8_t *excl, int32_t *phi,
                            float *d2, int k, int rmax, double rho, uint32_t key0, uint32_t key1,
                            uint32_t tag_base, uint32_t clip, int rs_mode, int sub_sweeps)
{
    size_t V = (size_t)W * H * T;
    ann_ctx a = {x, W, H, T, C, target, dtilde, excl, 0, 0};
    const uint8_t *mine = own ? own : target;
    int32_t *phi_old = (int32_t *)malloc(V * 3 * sizeof(int32_t));
    double *w = widen(d2, V);
    if (!phi_old || !w) {
        free(phi_old);
        free(w);
        return -1;
    }
    for (int j = 0; j < sub_sweeps; ++j) {
        memcpy(phi_old, phi, V * 3 * sizeof(int32_t));
        for (size_t p = 0; p < V; ++p)
            if (mine[p])
                propagate_one(&a, p, k, phi_old, phi, w);
    }
    for (size_t p = 0; p < V; ++p)
        if (mine[p])
            random_search_one(&a, p, k, rmax, rho, rs_mode, key0, key1, tag_base, clip, phi, w);
    narrow(w, d2, V);
    free(phi_old);
    free(w);
    return a.evals;
}

long long vio_ann(const float *x, int W, int H, int T, int C,
                  const uint8_t *target, const uint8_t *dtilde, const uint8_t *excl,
                  int32_t *phi, float *d2, int n_pm, int schedule, int rmax, double rho,
                  uint32_t key0, uint32_t key1, uint32_t tag_base, uint32_t clip)
{
    return vio_ann2(x, W, H, T, C, target, dtilde, excl, phi, d2, n_pm, schedule, rmax, rho, key0, key1,
                    tag_base, clip, 0, 1);
}

/* Exhaustive nearest neighbour over D~ in FP32 (ties: first source in
 * lexicographic order), for checking the approximate search. */
void vio_bruteforce_nn(const float *x, int W, int H, int T, int C,
                       const uint8_t *target, const uint8_t *dtilde, const uint8_t *excl,
                       int32_t *phi, float *d2)
{
    size_t V = (size_t)W * H * T;
    for (size_t p = 0; p < V; ++p) {
        if (!target[p])
            continue;
        int px, py, pt;
        coords(p, W, H, &px, &py, &pt);
        float bd = INFINITY;
        int b[3] = {0, 0, 0};
        for (size_t s = 0; s < V; ++s) {
            if (!dtilde[s])
                continue;
            int sx, sy, st;
            coords(s, W, H, &sx, &sy, &st);
            float d = vio_dist_f32(x, W, H, T, C, px, py, pt, sx, sy, st, excl);
            if (d < bd) {
                bd = d;
                b[0] = sx - px; b[1] = sy - py; b[2] = st - pt;
            }
        }
        phi[3 * p] = b[0]; phi[3 * p + 1] = b[1]; phi[3 * p + 2] = b[2];
        d2[p] = bd;
    }
}

/* ------------------------------------------------------------------------
 * Reconstruction, Eq. 4 and Eq. 5 (and Eq. 9 for the texture channels, Eq. 12
 * during the initialisation). For each voxel p with vote[p] = 1:
 *   Q = {q in N_p inside the video : allowed[q], d2[q] finite}
 *   sigma_p^2 = 75th percentile of {d2[q]} (nearest rank: the element of rank
 *     ceil(0.75 |Q|) in ascending order), the square of the 75th percentile of
 *     the distances d, since squaring is monotone;
 *   s_q = exp(-d2[q] / (2 sigma_p^2)) (weighted = 1) or 1 (weighted = 0); for
 *     sigma_p = 0 the limit: 1 where d2[q] = 0, else 0;
 *   x(p) = sum_q s_q x(p + phi(q)) / sum_q s_q, for every channel.
 * Reads x_in, writes x_out (voxels not voted are copied). A voxel with empty Q
 * is left unchanged and flagged in deferred[] (may be NULL). Returns the sum
 * over voted voxels of |x_out - x_in| over the first n_diff channels (the
 * numerator of the stopping criterion e of Sec. 3.7).
 * ---------------------------------------------------------------------- */
static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

static double vote_core(const float *x_in, float *x_out, int W, int H, int T, int C,
                        const uint8_t *vote, const uint8_t *allowed, const int32_t *phi,
                        const double *d2, int weighted, int n_diff, uint8_t *deferred)
{
    size_t V = (size_t)W * H * T;
    memcpy(x_out, x_in, V * (size_t)C * sizeof(float));
    double change = 0.0;
    double dq[NPATCH], sorted[NPATCH];
    size_t srcv[NPATCH];
    for (size_t p = 0; p < V; ++p) {
        if (deferred)
            deferred[p] = 0;
        if (!vote[p])
            continue;
        int px, py, pt;
        coords(p, W, H, &px, &py, &pt);
        int n = 0;
        for (int dt = -R; dt <= R; ++dt)
            for (int dy = -R; dy <= R; ++dy)
                for (int dx = -R; dx <= R; ++dx) {
                    int qx = px + dx, qy = py + dy, qt = pt + dt;
                    if (!inside(qx, qy, qt, W, H, T))
                        continue;
                    size_t q = vidx(qx, qy, qt, W, H);
                    if (!allowed[q] || !isfinite(d2[q]))
                        continue;
                    dq[n] = d2[q];
                    srcv[n] = vidx(px + phi[3 * q], py + phi[3 * q + 1], pt + phi[3 * q + 2], W, H);
                    ++n;
                }
        if (n == 0) {
            if (deferred)
                deferred[p] = 1;
            continue;
        }
        double sigma2 = 0.0;
        if (weighted) {
            memcpy(sorted, dq, (size_t)n * sizeof(double));
            qsort(sorted, (size_t)n, sizeof(double), cmp_double);
            int rank = (3 * n + 3) / 4;           /* ceil(0.75 n) */
            sigma2 = sorted[rank - 1];
        }
        double num[8] = {0}, den = 0.0;
        for (int i = 0; i < n; ++i) {
            double s;
            if (!weighted)
                s = 1.0;
            else if (sigma2 > 0.0)
                s = exp(-dq[i] / (2.0 * sigma2));
            else
                s = (dq[i] == 0.0) ? 1.0 : 0.0;
            den += s;
            for (int c = 0; c < C && c < 8; ++c)
                num[c] += s * (double)x_in[srcv[i] * (size_t)C + c];
        }
        for (int c = 0; c < C; ++c) {
            float v = (float)(num[c] / den);
            if (c < n_diff)
                change += fabs((double)v - (double)x_in[p * (size_t)C + c]);
            x_out[p * (size_t)C + c] = v;
        }
    }
    return change;
}

double vio_vote(const float *x_in, float *x_out, int W, int H, int T, int C,
                const uint8_t *vote, const uint8_t *allowed, const int32_t *phi,
                const float *d2, int weighted, int n_diff, uint8_t *deferred)
{
    size_t V = (size_t)W * H * T;
    double *w = widen(d2, V);
    if (!w)
        return NAN;
    double r = vote_core(x_in, x_out, W, H, T, C, vote, allowed, phi, w, weighted, n_diff, deferred);
    free(w);
    return r;
}

/* The vote with distances in double (the FP64 reference). */
double vio_vote_f64(const float *x_in, float *x_out, int W, int H, int T, int C,
                    const uint8_t *vote, const uint8_t *allowed, const int32_t *phi,
                    const double *d2, int weighted, int n_diff, uint8_t *deferred)
{
    return vote_core(x_in, x_out, W, H, T, C, vote, allowed, phi, d2, weighted, n_diff, deferred);
}

/* Final reconstruction, Eq. 6: p in H takes the value of its best contributor,
 * u(p + phi(q*)) with q* = argmin over q in N_p of d2[q] (ties: the first q in
 * the patch order dt, dy, dx ascending). */
static void final_core(const float *x_in, float *x_out, int W, int H, int T, int C,
                       const uint8_t *hole, const int32_t *phi, const double *d2)
{
    size_t V = (size_t)W * H * T;
    memcpy(x_out, x_in, V * (size_t)C * sizeof(float));
    for (size_t p = 0; p < V; ++p) {
        if (!hole[p])
            continue;
        int px, py, pt;
        coords(p, W, H, &px, &py, &pt);
        double bd = INFINITY;
        long long best = -1;
        for (int dt = -R; dt <= R; ++dt)
            for (int dy = -R; dy <= R; ++dy)
                for (int dx = -R; dx <= R; ++dx) {
                    int qx = px + dx, qy = py + dy, qt = pt + dt;
                    if (!inside(qx, qy, qt, W, H, T))
                        continue;
                    size_t q = vidx(qx, qy, qt, W, H);
                    if (best < 0 || d2[q] < bd) {
                        bd = d2[q];
                        best = (long long)q;
                    }
                }
        size_t q = (size_t)best;
        size_t s = vidx(px + phi[3 * q], py + phi[3 * q + 1], pt + phi[3 * q + 2], W, H);
        for (int c = 0; c < C; ++c)
            x_out[p * (size_t)C + c] = x_in[s * (size_t)C + c];
    }
}

void vio_final(const float *x_in, float *x_out, int W, int H, int T, int C,
               const uint8_t *hole, const int32_t *phi, const float *d2)
{
    double *w = widen(d2, (size_t)W * H * T);
    if (!w)
        return;
    final_core(x_in, x_out, W, H, T, C, hole, phi, w);
    free(w);
}

void vio_final_f64(const float *x_in, float *x_out, int W, int H, int T, int C,
                   const uint8_t *hole, const int32_t *phi, const double *d2)
{
    final_core(x_in, x_out, W, H, T, C, hole, phi, d2);
}

/* Energy, Eq. 1, evaluated in FP64: E_H = sum over p in H of d^2(W_p,
 * W_{p+phi(p)}), and the same sum over H~. */
void vio_energy(const float *x, int W, int H, int T, int C, const uint8_t *hole,
                const uint8_t *htilde, const int32_t *phi, double *out)
{
    size_t V = (size_t)W * H * T;
    double eh = 0.0, eht = 0.0;
    for (size_t p = 0; p < V; ++p) {
        if (!htilde[p])
            continue;
        int px, py, pt;
        coords(p, W, H, &px, &py, &pt);
        double d = vio_dist_f64(x, W, H, T, C, px, py, pt, px + phi[3 * p], py + phi[3 * p + 1],
                                pt + phi[3 * p + 2], NULL);
        eht += d;
        if (hole[p])
            eh += d;
    }
    out[0] = eh;
    out[1] = eht;
}
