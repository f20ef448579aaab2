// vi_device.cuh -- device-side building blocks shared by the kernels of the
// library: voxel indexing, the packed shift, Philox4x32-10 and the patch
// distance of Eq. 2 / Eq. 7b / Eq. 11.
#pragma once

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
// when C = 3), channel c4 in x1 (C = 5 only).
struct LevelView {
    int W, H, T;
    int HW;          // W * H
    int V;           // W * H * T  (< 2^31)
    float4 *x4;
    float *x1;
    uint8_t *code;
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

// Squared patch distance between the 5x5x5 patch of target p = (px, py, pt)
// and the patch of source s (linear index; its patch lies inside the video).
// Terms are summed in the patch's fixed order (dt, dy, dx ascending, then
// channels c0..c4), each (a - b)^2 added with one fused multiply-add, and the
// sum divided by N = 125 (Eq. 2 / 7b). Target voxels outside the video add
// nothing. With excl != nullptr, voxels r with excl[r] != 0 are left out too
// and the sum is divided by their complement's count (Eq. 11), +inf if empty.
template <bool C5>
__device__ __forceinline__ void acc_voxel(const LevelView &L, int r, int s, float &acc)
{
    const float4 a = __ldg(L.x4 + r);
    const float4 b = __ldg(L.x4 + s);
    float df;
    df = __fsub_rn(a.x, b.x); acc = __fmaf_rn(df, df, acc);
    df = __fsub_rn(a.y, b.y); acc = __fmaf_rn(df, df, acc);
    df = __fsub_rn(a.z, b.z); acc = __fmaf_rn(df, df, acc);
    df = __fsub_rn(a.w, b.w); acc = __fmaf_rn(df, df, acc);
    if (C5) {
        df = __fsub_rn(__ldg(L.x1 + r), __ldg(L.x1 + s));
        acc = __fmaf_rn(df, df, acc);
    }
}

template <bool C5>
__device__ __forceinline__ float patch_d2_interior(const LevelView &L, int p, int s)
{
    const int W = L.W, HW = L.HW;
    const int off = 2 + 2 * W + 2 * HW;
    const int rb = p - off, sb = s - off;
    float acc = 0.0f;
#pragma unroll 1
    for (int dt = 0; dt < 5; ++dt) {
#pragma unroll
        for (int dy = 0; dy < 5; ++dy) {
            const int ro = rb + dt * HW + dy * W;
            const int so = sb + dt * HW + dy * W;
#pragma unroll
            for (int dx = 0; dx < 5; ++dx)
                acc_voxel<C5>(L, ro + dx, so + dx, acc);
        }
    }
    return __fdiv_rn(acc, 125.0f);
}

template <bool C5>
__device__ float patch_d2_general(const LevelView &L, int px, int py, int pt, int s,
                                  const uint8_t *excl)
{
    const int W = L.W, HW = L.HW;
    float acc = 0.0f;
    int n = 0;
    for (int dt = -2; dt <= 2; ++dt) {
        const int rt = pt + dt;
        if ((unsigned)rt >= (unsigned)L.T)
            continue;
        for (int dy = -2; dy <= 2; ++dy) {
            const int ry = py + dy;
            if ((unsigned)ry >= (unsigned)L.H)
                continue;
            for (int dx = -2; dx <= 2; ++dx) {
                const int rx = px + dx;
                if ((unsigned)rx >= (unsigned)W)
                    continue;
                const int r = rt * HW + ry * W + rx;
                if (excl && excl[r])
                    continue;
                acc_voxel<C5>(L, r, s + dt * HW + dy * W + dx, acc);
                ++n;
            }
        }
    }
    if (excl) {
        if (n == 0)
            return __int_as_float(0x7f800000);
        return __fdiv_rn(acc, (float)n);
    }
    return __fdiv_rn(acc, 125.0f);
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
