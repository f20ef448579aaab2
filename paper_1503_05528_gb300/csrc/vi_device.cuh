// vi_device.cuh -- device-side building blocks shared by the kernels of the
// library: voxel indexing, the packed shift, Philox4x32-10 and the patch
// distance of Eq. 2 / Eq. 7b / Eq. 11.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace vi {

// Per-voxel set codes (Sec. 2): H, H~ (targets), D~ (sources).
enum : uint8_t { CODE_HOLE = 1, CODE_TARGET = 2, CODE_SOURCE = 4 };

// A shift phi(p) = (dx, dy, dt), 8 bytes, read and written as one 64-bit word.
struct __align__(8) Shift {
    short dx, dy, dt, pad;
};

// One pyramid level as the kernels see it. Channels c0..c3 live in x4 (c3 = 0
// when C = 3), channel c4 in x1 (C = 5 only). With FP16 storage, h4 holds
// channels c0..c3 rounded to FP16 (four halves per uint2) and hmax[c] bounds
// |x_c| over every value the level has held (float bits, raised with
// atomicMax); h4 == nullptr means FP32 storage only.
struct LevelView {
    int W, H, T;
    int HW;          // W * H
    int V;           // W * H * T  (< 2^31)
    float4 *x4;
    float *x1;
    uint8_t *code;
    uint2 *h4;
    unsigned *hmax;
};

__device__ __forceinline__ void decode(int p, int W, int HW, int &x, int &y, int &t)
{
    t = p / HW;
    int r = p - t * HW;
    y = r / W;
    x = r - y * W;
}

__device__ __forceinline__ bool inside(const LevelView &L, int x, int y, int t)
{
    return (unsigned)x < (unsigned)L.W && (unsigned)y < (unsigned)L.H && (unsigned)t < (unsigned)L.T;
}

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64-bit
// multiplies by the Philox constants, mixing the high halves with the other
// two words and the round key; the key advances by the Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// floor(r_max * rho^k * delta) for delta = (2*(w >> 8) + 1 - 2^24) / 2^24 in
// (-1, 1) and rho = 2^-m, as exact integer arithmetic: the product
// r_max * (2*(w >> 8) + 1 - 2^24) shifted right (floor) by m*k + 24 bits.
__device__ __forceinline__ int random_offset(uint32_t w, int rmax, int shift)
{
    const long long delta_int = 2ll * (long long)(w >> 8) + 1ll - (1ll << 24);
    const long long prod = (long long)rmax * delta_int;
    return (int)(prod >> (shift < 63 ? shift : 63));
}

// Index in [0, n) from one word: floor(w * n / 2^32).
__device__ __forceinline__ uint32_t uniform_index(uint32_t w, uint32_t n)
{
    return (uint32_t)(((unsigned long long)w * (unsigned long long)n) >> 32);
}

// ---------------------------------------------------------------------------
// Squared patch distance between the 5x5x5 patch of target p = (px, py, pt)
// and the patch of source s (linear index; its patch lies inside the video),
// Eq. 2 / 7b. Target voxels outside the video add nothing; the sum is divided
// by N = 125. With excl != nullptr, voxels r with excl[r] != 0 are left out
// too and the sum is divided by the count of voxels kept (Eq. 11), +inf if
// none.
//
// Summation order (the oracle uses the same): the terms (a - b)^2 of one row
// (fixed dt, dy; dx ascending, channels c0..c4) are accumulated by fused
// multiply-adds starting from 0; the 5 row sums of a slice (fixed dt) are
// added in dy order; the 5 slice sums are added in dt order. The five row
// chains of a slice are independent, so a thread keeps 25 voxel loads and
// five FMA chains in flight rather than one serial chain of 625 terms.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float half_lo(unsigned u) { return __half2float(__ushort_as_half((unsigned short)(u & 0xFFFFu))); }
__device__ __forceinline__ float half_hi(unsigned u) { return __half2float(__ushort_as_half((unsigned short)(u >> 16))); }

// Adds the terms of voxel pair (r, s) to acc: from the FP32 channels, or with
// H from the FP16 copies of c0..c3 (converted exactly to FP32).
template <bool C5, bool H = false>
__device__ __forceinline__ void acc_voxel(const LevelView &L, int r, int s, float &acc)
{
    static_assert(!(C5 && H), "the FP16 copy holds channels c0..c3 only");
    float a0, a1, a2, a3, b0, b1, b2, b3;
    if (H) {
        const uint2 ua = __ldg(L.h4 + r), ub = __ldg(L.h4 + s);
        a0 = half_lo(ua.x); a1 = half_hi(ua.x); a2 = half_lo(ua.y); a3 = half_hi(ua.y);
        b0 = half_lo(ub.x); b1 = half_hi(ub.x); b2 = half_lo(ub.y); b3 = half_hi(ub.y);
    } else {
        const float4 a = __ldg(L.x4 + r);
        const float4 b = __ldg(L.x4 + s);
        a0 = a.x; a1 = a.y; a2 = a.z; a3 = a.w;
        b0 = b.x; b1 = b.y; b2 = b.z; b3 = b.w;
    }
    float df;
    df = __fsub_rn(a0, b0); acc = __fmaf_rn(df, df, acc);
    df = __fsub_rn(a1, b1); acc = __fmaf_rn(df, df, acc);
    df = __fsub_rn(a2, b2); acc = __fmaf_rn(df, df, acc);
    df = __fsub_rn(a3, b3); acc = __fmaf_rn(df, df, acc);
    if (C5) {
        df = __fsub_rn(__ldg(L.x1 + r), __ldg(L.x1 + s));
        acc = __fmaf_rn(df, df, acc);
    }
}

// Sum of one whole slice: ro, so = target / source voxel of offset (-2, -2).
template <bool C5, bool H = false>
__device__ __forceinline__ float slice_sum(const LevelView &L, int ro, int so)
{
    float r[5];
#pragma unroll
    for (int dy = 0; dy < 5; ++dy) {
        r[dy] = 0.0f;
#pragma unroll
        for (int dx = 0; dx < 5; ++dx)
            acc_voxel<C5, H>(L, ro + dy * L.W + dx, so + dy * L.W + dx, r[dy]);
    }
    float s = r[0];
#pragma unroll
    for (int dy = 1; dy < 5; ++dy)
        s = __fadd_rn(s, r[dy]);
    return s;
}

template <bool C5>
__device__ __forceinline__ float patch_d2_interior(const LevelView &L, int p, int s)
{
    const int W = L.W, HW = L.HW;
    const int off = 2 + 2 * W + 2 * HW;
    const int rb = p - off, sb = s - off;
    float total = 0.0f;
#pragma unroll 1
    for (int dt = 0; dt < 5; ++dt)
        total = __fadd_rn(total, slice_sum<C5>(L, rb + dt * HW, sb + dt * HW));
    return __fdiv_rn(total, 125.0f);
}

// The same distance for a candidate that only matters if it beats the current
// best d (an interior target, full distance): after every slice the running
// total is compared with thr = 125 * best rounded up, and the evaluation stops
// as soon as the total reaches it, returning +inf. The terms are non-negative,
// so the total only grows, and dividing by 125 preserves order: a stopped
// candidate's full distance is >= best, so it would not have been accepted. A
// completed evaluation returns exactly patch_d2_interior's value. `gathered`
// counts the source voxels read.
template <bool C5>
__device__ __forceinline__ float patch_d2_interior_bounded(const LevelView &L, int p, int s, float best,
                                                           unsigned &gathered)
{
    const int W = L.W, HW = L.HW;
    const int off = 2 + 2 * W + 2 * HW;
    const int rb = p - off, sb = s - off;
    const float thr = __fmul_ru(best, 125.0f);
    float total = 0.0f;
#pragma unroll 1
    for (int dt = 0; dt < 5; ++dt) {
        total = __fadd_rn(total, slice_sum<C5>(L, rb + dt * HW, sb + dt * HW));
        gathered += 25;
        if (total >= thr)
            return __int_as_float(0x7f800000);
    }
    return __fdiv_rn(total, 125.0f);
}

template <bool C5, bool H = false>
__device__ __forceinline__ float slice_general(const LevelView &L, int px, int py, int pt, int s, int dt,
                                               const uint8_t *excl, int &n);

// Targets near the border (clipped patch) and the partial distance of Eq. 11.
template <bool C5>
__device__ float patch_d2_general(const LevelView &L, int px, int py, int pt, int s,
                                  const uint8_t *excl, unsigned *gathered = nullptr)
{
    float total = 0.0f;
    int n = 0;
#pragma unroll 1
    for (int dt = -2; dt <= 2; ++dt) {
        int sn;
        total = __fadd_rn(total, slice_general<C5>(L, px, py, pt, s, dt, excl, sn));
        n += sn;
    }
    if (gathered)
        *gathered += (unsigned)n;
    if (excl) {
        if (n == 0)
            return __int_as_float(0x7f800000);
        return __fdiv_rn(total, (float)n);
    }
    return __fdiv_rn(total, 125.0f);
}

// acc_voxel for a voxel that may be skipped: both loads are issued from valid
// addresses; a skipped voxel adds fma(0, 0, acc) = acc exactly.
template <bool C5>
__device__ __forceinline__ void acc_voxel_if(const LevelView &L, int r, int s, bool use, float &acc)
{
    const float4 a = __ldg(L.x4 + r);
    const float4 b = __ldg(L.x4 + s);
    float df;
    df = use ? __fsub_rn(a.x, b.x) : 0.0f; acc = __fmaf_rn(df, df, acc);
    df = use ? __fsub_rn(a.y, b.y) : 0.0f; acc = __fmaf_rn(df, df, acc);
    df = use ? __fsub_rn(a.z, b.z) : 0.0f; acc = __fmaf_rn(df, df, acc);
    df = use ? __fsub_rn(a.w, b.w) : 0.0f; acc = __fmaf_rn(df, df, acc);
    if (C5) {
        const float a1 = __ldg(L.x1 + r), b1 = __ldg(L.x1 + s);
        df = use ? __fsub_rn(a1, b1) : 0.0f;
        acc = __fmaf_rn(df, df, acc);
    }
}

// One slice (fixed dt offset in [-2, 2]) of a clipped or partial distance:
// the row sums over in-video, non-excluded target voxels, added in dy order;
// n receives the number of voxels used.
template <bool C5, bool H>
__device__ __forceinline__ float slice_general(const LevelView &L, int px, int py, int pt, int s, int dt,
                                               const uint8_t *excl, int &n)
{
    const int W = L.W, HW = L.HW;
    const int rt = pt + dt;
    float slice = 0.0f;
    n = 0;
    for (int dy = -2; dy <= 2; ++dy) {
        const int ry = py + dy;
        float row = 0.0f;
        if ((unsigned)rt < (unsigned)L.T && (unsigned)ry < (unsigned)L.H) {
            for (int dx = -2; dx <= 2; ++dx) {
                const int rx = px + dx;
                if ((unsigned)rx >= (unsigned)W)
                    continue;
                const int r = rt * HW + ry * W + rx;
                if (excl && excl[r])
                    continue;
                acc_voxel<C5, H>(L, r, s + dt * HW + dy * W + dx, row);
                ++n;
            }
        }
        slice = __fadd_rn(slice, row);
    }
    return slice;
}

// The same slice, fully unrolled and predicated, so that its 25 voxel loads
// are independent (a skipped target voxel reads the source voxel instead and
// contributes nothing). Used for the partial distance, where any voxel may
// be excluded.
template <bool C5>
__device__ __forceinline__ float slice_masked(const LevelView &L, int px, int py, int pt, int s, int dt,
                                              const uint8_t *excl, int &n)
{
    const int W = L.W, HW = L.HW;
    const int rt = pt + dt;
    const bool t_ok = (unsigned)rt < (unsigned)L.T;
    float slice = 0.0f;
    n = 0;
#pragma unroll
    for (int dy = -2; dy <= 2; ++dy) {
        const int ry = py + dy;
        const bool y_ok = t_ok && (unsigned)ry < (unsigned)L.H;
        float row = 0.0f;
#pragma unroll
        for (int dx = -2; dx <= 2; ++dx) {
            const int rx = px + dx;
            const int sv = s + dt * HW + dy * W + dx;
            bool use = y_ok && (unsigned)rx < (unsigned)W;
            const int r = use ? rt * HW + ry * W + rx : sv;
            if (excl)
                use = use && !excl[r];
            acc_voxel_if<C5>(L, r, sv, use, row);
            n += use ? 1 : 0;
        }
        slice = __fadd_rn(slice, row);
    }
    return slice;
}

// The distance computed by a group of G lanes (G = 1, 2, 4 or 8 consecutive
// lanes of a warp; gmask is the group's lane mask, sub the lane's rank in it).
// Lane sub gathers the slices dt = sub, sub + G, ...; the group adds the slice
// sums in dt order with shuffles, so every lane holds the same total, in the
// same order as patch_d2_interior / patch_d2_general: the value is bit-
// identical for every G. Slices are gathered in rounds of G; after each round
// the running total is compared with 125 * best rounded up (the full-distance
// case only) and the evaluation stops as soon as it is reached, returning +inf
// (the total only grows, so the candidate could not win). best = +inf gives
// the unbounded distance. `gathered` counts the source voxels this lane read.
// PARTIAL selects the distance of Eq. 11 (excl = H', every voxel tested).
// Otherwise excl is ignored; a target whose patch stays inside the frame
// (x and y at least 2 from the border) takes the unrolled slice_sum for each
// slice inside the video and adds 0 for a slice outside it (the same terms,
// in the same order, as slice_general).
template <bool C5, int G, bool PARTIAL>
__device__ __forceinline__ float group_d2(const LevelView &L, int p, int px, int py, int pt, int s,
                                          const uint8_t *excl, float best, int sub, unsigned gmask,
                                          unsigned &gathered)
{
    const int HW = L.HW;
    const int off = 2 + 2 * L.W + 2 * HW;
    const bool frame_inside = px >= 2 && px < L.W - 2 && py >= 2 && py < L.H - 2;
    const float thr = __fmul_ru(best, 125.0f);
    float total = 0.0f;
    int n = 0;
#pragma unroll 1
    for (int r0 = 0; r0 < 5; r0 += G) {
        const int dt = r0 + sub;
        float mine = 0.0f;
        int my_n = 0;
        if (dt < 5) {
            if (PARTIAL) {
                mine = slice_masked<C5>(L, px, py, pt, s, dt - 2, excl, my_n);
            } else if (frame_inside) {
                if ((unsigned)(pt + dt - 2) < (unsigned)L.T) {
                    mine = slice_sum<C5>(L, p - off + dt * HW, s - off + dt * HW);
                    my_n = 25;
                }
            } else {
                mine = slice_general<C5>(L, px, py, pt, s, dt - 2, nullptr, my_n);
            }
            gathered += (unsigned)my_n;
        }
#pragma unroll
        for (int j = 0; j < G; ++j) {
            if (r0 + j < 5) {
                total = __fadd_rn(total, G == 1 ? mine : __shfl_sync(gmask, mine, j, G));
                if (PARTIAL)
                    n += G == 1 ? my_n : __shfl_sync(gmask, my_n, j, G);
            }
        }
        if (!PARTIAL && total >= thr)
            return __int_as_float(0x7f800000);
    }
    if (PARTIAL) {
        if (n == 0)
            return __int_as_float(0x7f800000);
        return __fdiv_rn(total, (float)n);
    }
    return __fdiv_rn(total, 125.0f);
}

// FP16 copy of voxel v's channels c0..c3 (FP16 storage: L.h4 != nullptr),
// and hmax raised to cover the values written. hmax holds |x| as float bits, so
// unsigned comparison orders it (a NaN compares above +inf and disables the
// screening below).
__device__ __forceinline__ unsigned pack_half2(float lo, float hi)
{
    return (unsigned)__half_as_ushort(__float2half_rn(lo)) |
           ((unsigned)__half_as_ushort(__float2half_rn(hi)) << 16);
}

__device__ __forceinline__ unsigned abs_bits(float x) { return __float_as_uint(x) & 0x7fffffffu; }

__device__ __forceinline__ void raise_hmax(unsigned *hmax, int c, unsigned m)
{
    if (m > __ldcg(hmax + c))
        atomicMax(hmax + c, m);
}

__device__ __forceinline__ void shadow_store(const LevelView &L, int v, float4 a)
{
    L.h4[v] = make_uint2(pack_half2(a.x, a.y), pack_half2(a.z, a.w));
}

// shadow_store for one voxel written by a single thread, hmax raised at once.
__device__ __forceinline__ void shadow_store_raise(const LevelView &L, int v, float4 a)
{
    shadow_store(L, v, a);
    raise_hmax(L.hmax, 0, abs_bits(a.x));
    raise_hmax(L.hmax, 1, abs_bits(a.y));
    raise_hmax(L.hmax, 2, abs_bits(a.z));
    raise_hmax(L.hmax, 3, abs_bits(a.w));
}

// ---------------------------------------------------------------------------
// FP16 screening (storage = 1). A candidate's FP32 distance is only computed
// when its distance over the FP16 copies does not already prove that it
// cannot beat the current best; the FP32 comparison then decides, so the
// shift maps are the same bit for bit as with FP32 storage.
//
// The proof. Over the k voxels summed so far let x be the vector of FP32
// differences in channels c0..c3 and x' that of the FP16 copies' differences,
// S = |x|^2, S' = |x'|^2. Rounding to FP16 moves a value v with |v| <= M_c by
// at most 2^-11 |v| + 2^-25, so every entry of e = x' - x is at most
// delta_c = 2^-10 M_c + 2^-24 in channel c, and |e| <= sqrt(k * D) with
// D = sum_c delta_c^2. By the triangle inequality sqrt(S) >= sqrt(S') -
// sqrt(k D), and the full sum S_full (all voxels, all channels: the terms are
// non-negative) is at least S. The FP32 path
// accepts only when fl(fl(S_full) / 125) < best; its summation (at most 37
// roundings of non-negative terms) is within a factor 1 - 2^-18 of S_full, so
// S_full >= 125 best (1 + 2^-16) rules acceptance out. The bound is evaluated
// with directed rounding (the computed S' shrunk by 2^-17 for its own
// rounding, square roots and the subtraction rounded down, the right-hand
// side rounded up), so every approximation errs towards passing. An M_c that
// is not finite or exceeds the FP16 range makes D infinite or NaN and every
// candidate passes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float screen_d2bound(const LevelView &L)
{
    float D = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float m = __uint_as_float(__ldg(L.hmax + c));
        const float dl = (m <= 65504.0f) ? __fadd_ru(__fmul_ru(m, 0x1p-10f), 0x1p-24f)
                                          : __int_as_float(0x7f800000);
        D = __fadd_ru(D, __fmul_ru(dl, dl));
    }
    return D;
}

// True when the candidate must be rescored in FP32 (see above); D from
// screen_d2bound over channels c0..c3. The screen reads only the four
// channels of h4 (one 8-byte load per voxel): leaving channel c4 out can only
// lower S, so the bound stays valid, and a candidate costs half the load
// instructions of the FP32 distance. Slices are summed in rounds of G as in
// group_d2 and the test runs after every round; every lane of the group
// holds the same totals and takes the same decision. `gathered` counts the
// FP16 source voxels read.
template <bool C5, int G>
__device__ __forceinline__ bool group_screen(const LevelView &L, int p, int px, int py, int pt, int s,
                                             float best, float D, int sub, unsigned gmask, unsigned &gathered)
{
    const int HW = L.HW;
    const int off = 2 + 2 * L.W + 2 * HW;
    const bool frame_inside = px >= 2 && px < L.W - 2 && py >= 2 && py < L.H - 2;
    const float rhs = __fsqrt_ru(__fmul_ru(best, 125.0019073486328125f));   // 125 (1 + 2^-16)
    float total = 0.0f;
#pragma unroll 1
    for (int r0 = 0; r0 < 5; r0 += G) {
        const int dt = r0 + sub;
        float mine = 0.0f;
        if (dt < 5) {
            int my_n = 0;
            if (frame_inside) {
                if ((unsigned)(pt + dt - 2) < (unsigned)L.T) {
                    mine = slice_sum<false, true>(L, p - off + dt * HW, s - off + dt * HW);
                    my_n = 25;
                }
            } else {
                mine = slice_general<false, true>(L, px, py, pt, s, dt - 2, nullptr, my_n);
            }
            gathered += (unsigned)my_n;
        }
#pragma unroll
        for (int j = 0; j < G; ++j)
            if (r0 + j < 5)
                total = __fadd_rn(total, G == 1 ? mine : __shfl_sync(gmask, mine, j, G));
        const int k = 25 * (r0 + G < 5 ? r0 + G : 5);   // voxels summed so far, at most
        const float lower = __fsub_rd(__fsqrt_rd(__fmul_rd(total, 0.999992370605468750f)),   // 1 - 2^-17
                                      __fsqrt_ru(__fmul_ru((float)k, D)));
        if (lower >= rhs)
            return false;
    }
    return true;
}

template <bool C5>
__device__ __forceinline__ float patch_d2(const LevelView &L, int p, int px, int py, int pt, int s,
                                          const uint8_t *excl)
{
    const bool interior = px >= 2 && px < L.W - 2 && py >= 2 && py < L.H - 2 && pt >= 2 &&
                          pt < L.T - 2;
    if (interior && excl == nullptr)
        return patch_d2_interior<C5>(L, p, s);
    return patch_d2_general<C5>(L, px, py, pt, s, excl);
}

// Index of the segment holding global index i: prefix[c] <= i < prefix[c+1]
// (prefix has n + 1 ascending entries; batches of clips).
__device__ __forceinline__ int find_segment(const int *__restrict__ prefix, int n, int i)
{
    int lo = 0, hi = n;   // invariant: prefix[lo] <= i < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= i)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void count_evals(unsigned long long *ctr, unsigned n)
{
    // one atomic per warp
    unsigned tot = __reduce_add_sync(0xffffffffu, n);
    if ((threadIdx.x & 31) == 0 && tot)
        atomicAdd(ctr, (unsigned long long)tot);
}

}  // namespace vi
