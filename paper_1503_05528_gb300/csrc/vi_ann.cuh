// vi_ann.cuh -- the PatchMatch step of Sec. 3.1 (Algorithm 1) as a parallel
// (Jacobi) sweep: candidate generation, exact pruning, lane groups and, with
// FP16 storage, the screening of a candidate before its FP32 distance.
//
// One group of G lanes per target voxel. Targets are raster ordered, so a warp
// covers a run of neighbouring voxels along x; with the piecewise-constant
// shift maps PatchMatch relies on, their candidate source patches are
// neighbours too, and the 5x5x5 gathers of a warp coalesce into contiguous
// rows. vi_search.cu instantiates the FP32-storage kernels and vi_search_h.cu
// the FP16-storage ones, so the two compile in parallel.
#pragma once

#include "vi_launch.h"

namespace vi {

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

inline int device_sms()
{
    static int sms = 0;
    if (sms <= 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 152;
    }
    return sms;
}

// Grid of a persistent batch launch: one wave of blocks of `block` threads
// (blocks_per_sm resident on every SM), or fewer when the work is smaller.
inline int persistent_grid(long long threads, int blocks_per_sm = 8, int block = 256)
{
    const long long cap = (long long)device_sms() * blocks_per_sm;
    const long long need = (threads + block - 1) / block;
    return (int)(need < 1 ? 1 : (need < cap ? need : cap));
}

// Threads per block of the step kernels. Smaller blocks' warps finish closer
// together (a target's work varies a lot: a rejected candidate costs one
// slice, an accepted one five), so the SM refills sooner. Per inpainting,
// 128 threads against 256: 22.9 against 23.4 ms (320x240x60) and 261
// against 276 ms (1280x720x100); 64 against 128, with the warp-shared step:
// 19.84 against 20.04 ms (320x240x60).
constexpr int STEP_BLOCK = 64;

// Resident blocks of 256 threads per SM the step kernels are compiled for
// (twice as many of STEP_BLOCK): the register budget per thread is
// 65536 / (256 * blocks). The step is a chain of
// dependent gathers that hit L1/L2, so loads in flight per thread matter more
// than warps: measured on the 320x240x60 workload (ms per inpainting, summed
// step launches; 4 / 3 / 2 blocks = 64 / 80 / 128 registers): G = 1
// 16.3 / 16.5 / 15.0, G = 2 5.5 / 4.6 / 4.2, G = 8 2.9 / 2.8 / 3.4, onion
// peel 1.4 / 1.3 / 1.3.
template <int G, bool PARTIAL>
constexpr int step_min_blocks()
{
    return (G == 8 && !PARTIAL) ? 3 : 2;
}

// Lanes per target: the smallest G in {1, 2, 4, 8} that gives the level at
// least 512 threads per SM. Measured on the 320x240x60 workload (one launch,
// microseconds, G = 1 / 2 / 4 / 8): 445k targets 280 / 301 / 447 / 681,
// 126k targets 101 / 108 / 147 / 207, 40k targets 79 / 51 / 60 / 82, 15k
// targets 78 / 46 / 37 / 34: more lanes pay only while the targets alone
// leave the SMs idle. The partial distance (onion peel, coarsest level, few
// targets) always uses G = 8.
inline int pick_group(int nT)
{
    const long long want = (long long)device_sms() * 512;
    int G = 1;
    while (G < 8 && (long long)nT * G < want)
        G *= 2;
    return G;
}

inline int blocks_for(long long n, int block)
{
    long long g = (n + block - 1) / block;
    return (int)(g < 1 ? 1 : g);
}

// Per-lane counts of one step launch.
struct StepCount {
    unsigned evals = 0;       // valid candidates (the oracle's count)
    unsigned gathered = 0;    // FP32 source voxels read
    unsigned gathered_h = 0;  // FP16 source voxels read
    unsigned screened = 0;    // candidates screened in FP16
    unsigned passed = 0;      // of those, rescored in FP32
};

// One candidate of Algorithm 1 for target p: counted as an evaluation when it
// lands in D~ (the oracle counts the same). A candidate equal to the current
// best shift, or to one already rejected in this iteration, has that shift's
// distance, which cannot be strictly smaller than the current best, so it is
// resolved without a gather. With F16 the candidate is first screened on the
// FP16 copies (group_screen): one that provably cannot beat the best is
// rejected there. Otherwise the G lanes of the group gather its FP32
// distance, bounded by the current best; the decision is the same bit for bit
// as with a full evaluation.
template <bool C5, int G, bool PARTIAL, bool F16>
__device__ __forceinline__ void try_candidate_g(const AnnArgs &a, int p, int px, int py, int pt, int s,
                                                int cdx, int cdy, int cdt, Shift &cur, float &d,
                                                Rejected &rej, float D, StepCount &n, int sub,
                                                unsigned gmask)
{
    if (s < 0)
        return;
    ++n.evals;
    const unsigned long long key = shift_key(cdx, cdy, cdt);
    if (key == shift_key(cur.dx, cur.dy, cur.dt) || rej.has(key))
        return;
    if (F16 && a.L.h4) {
        ++n.screened;
        if (!group_screen<C5, G>(a.L, p, px, py, pt, s, d, D, sub, gmask, n.gathered_h)) {
            rej.add(key);
            return;
        }
        ++n.passed;
    }
    const float dd = group_d2<C5, G, PARTIAL>(a.L, p, px, py, pt, s, a.excl, d, sub, gmask, n.gathered);
    if (dd < d) {
        d = dd;
        cur.dx = (short)cdx;
        cur.dy = (short)cdy;
        cur.dt = (short)cdt;
    } else {
        rej.add(key);
    }
}

// One PatchMatch iteration k for target i of the clip described by a, by the
// G lanes of one group: propagation from the three neighbours (Algorithm 1;
// sign by the parity of k), then the random search of Eq. 3 around the
// propagated shift. Reads phi_in / d_in (the state when iteration k began),
// writes phi_out / d_out. The three neighbours' shifts and their sources' set
// codes are loaded together before any distance.
template <bool C5, int G, bool PARTIAL, bool F16>
__device__ __forceinline__ void ann_one(const AnnArgs &a, int i, int k, int span, bool do_random, int sub,
                                        unsigned gmask, StepCount &n)
{
    const LevelView L = a.L;   // a register copy (the batch kernels read a from global memory)
    const float D = (F16 && L.h4) ? screen_d2bound(L) : 0.0f;
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
    // With FP16 storage only the random-search candidate is screened. A
    // neighbour's shift often wins (that is what propagation is for), and a
    // winner pays for the screen and the FP32 distance both; a random
    // candidate almost never wins. Measured on GB300 (full inpainting, ms per
    // clip): FP32 storage 38.0 (320x240x60) and 490 (1280x720x100); all four
    // candidates screened on five channels 52.6 and 661; the random one only,
    // screened on c0..c3, 39.4 and 462.
    //
    // A neighbour whose shift did not change since this target last judged
    // the same neighbour in the same direction (chg_span sweeps back: two with
    // one sweep per iteration; with sub-sweeps one within an iteration, and
    // the sub-sweeps of the iteration between plus one at its first) offers
    // the candidate this target already judged, on the same video (the
    // channels are fixed within an ANN call): then it either lost (its
    // distance was >= this target's distance, which has not grown since) or
    // won and has been kept or beaten since. Either way it cannot be strictly
    // better now, so it is counted and skipped without a gather; every
    // decision stays the same.
    Rejected rej;
    const unsigned span_mask = a.chg_in != nullptr && span > 0 ? (1u << span) - 1u : 0u;
    const bool st0 = span_mask && t0 && (a.chg_in[r0] & span_mask) == 0;
    const bool st1 = span_mask && t1 && (a.chg_in[r1] & span_mask) == 0;
    const bool st2 = span_mask && t2 && (a.chg_in[r2] & span_mask) == 0;
    const Shift start = cur;
    if (st0) {
        if (s0 >= 0)
            ++n.evals;
    } else {
        try_candidate_g<C5, G, PARTIAL, false>(a, p, px, py, pt, s0, c0.dx, c0.dy, c0.dt, cur, d, rej, D, n, sub,
                                               gmask);
    }
    if (st1) {
        if (s1 >= 0)
            ++n.evals;
    } else {
        try_candidate_g<C5, G, PARTIAL, false>(a, p, px, py, pt, s1, c1.dx, c1.dy, c1.dt, cur, d, rej, D, n, sub,
                                               gmask);
    }
    if (st2) {
        if (s2 >= 0)
            ++n.evals;
    } else {
        try_candidate_g<C5, G, PARTIAL, false>(a, p, px, py, pt, s2, c2.dx, c2.dy, c2.dt, cur, d, rej, D, n, sub,
                                               gmask);
    }

    // random search: Eq. 3 (one radius per k), or every radius rmax rho^i >= 1
    // around the best shift so far (counter word 3 = i)
    if (do_random) {
        for (int i = 0; i < 31; ++i) {
            const int sh = a.rs_mode ? a.rho_log2 * i : a.rho_log2 * k;
            if (a.rs_mode && (sh > 30 || (a.rmax >> sh) < 1))
                break;
            const uint4 w = philox4x32_10(make_uint4((uint32_t)p, a.tag | (uint32_t)k, a.clip,
                                                     a.rs_mode ? (uint32_t)i : 0u),
                                          a.key0, a.key1);
            const int cdx = cur.dx + random_offset(w.x, a.rmax, sh + 24);
            const int cdy = cur.dy + random_offset(w.y, a.rmax, sh + 24);
            const int cdt = cur.dt + random_offset(w.z, a.rmax, sh + 24);
            const int s3 = source_of(L, px, py, pt, cdx, cdy, cdt);
            try_candidate_g<C5, G, PARTIAL, F16>(a, p, px, py, pt, s3, cdx, cdy, cdt, cur, d, rej, D, n, sub,
                                                 gmask);
            if (!a.rs_mode)
                break;
        }
    }
    if (sub == 0) {
        a.phi_out[p] = cur;
        a.d_out[p] = d;
        if (a.chg_out) {
            const bool changed = cur.dx != start.dx || cur.dy != start.dy || cur.dt != start.dt;
            a.chg_out[p] = (uint8_t)((changed ? 1u : 0u) | ((unsigned)a.chg_in[p] << 1));
        }
    }
}

// ---------------------------------------------------------------------------
// Warp-shared lanes (lanes_per_target = 32). With one lane per target, a warp
// spends each candidate's gathers on the lanes whose candidate needs them
// (not rejected by a cheap test) while the others wait: at the largest
// levels about 13 of 32 lanes were active on average. Here lane l still owns
// target l of the warp's 32 (its state, counts and decisions), but every
// candidate that needs a distance is evaluated by a group of G lanes, G
// chosen per candidate round from how many lanes need one: the most lanes
// (at most 8) that still serve them all at once. A target's candidates keep
// their order (propagation from the three neighbours, then the random
// search), each bounded by the best distance so far, and group_d2 adds the
// slices in the same order for every G, so every decision and every output
// is the same as with a fixed G.
// ---------------------------------------------------------------------------

// The pending candidates of mask M (owner lanes), G lanes each: group j
// serves the owner holding the j-th set bit of M, with the owner's target,
// source and bound. Returns, on each owner lane, its candidate's bounded
// distance (group_d2). The gathers read the level's sizes and channel pointers
// from register copies (LevelView(L) here, and the copy ann_one_warp takes):
// the batch kernels find them in the clip's descriptor in global memory, and
// read through a reference they were reloaded inside the gather loop
// (measured on the 48-clip batch: step kernels 822 ms per batch with the
// copies, 931 ms without).
template <bool C5, int G>
__device__ __forceinline__ float warp_serve_d2(const LevelView &L, unsigned M, int lane, int p, int px, int py,
                                               int pt, int s, float best, unsigned &gathered)
{
    const unsigned FULL = 0xffffffffu;
    const int c = __popc(M);
    const int j = lane / G;
    const int o = j < c ? (int)__fns(M, 0, j + 1) : lane;
    const int op = __shfl_sync(FULL, p, o), opx = __shfl_sync(FULL, px, o), opy = __shfl_sync(FULL, py, o),
              opt = __shfl_sync(FULL, pt, o), os = __shfl_sync(FULL, s, o);
    const float ob = __shfl_sync(FULL, best, o);
    float dd = __int_as_float(0x7f800000);
    if (j < c)
        dd = group_d2<C5, G, false>(LevelView(L), op, opx, opy, opt, os, nullptr, ob, lane & (G - 1), group_mask<G>(),
                                    gathered);
    const int r = __popc(M & ((1u << lane) - 1u));
    return __shfl_sync(FULL, dd, (r * G) & 31);
}

template <bool C5>
__device__ __forceinline__ float warp_d2(const LevelView &L, unsigned M, int lane, int p, int px, int py, int pt,
                                         int s, float best, unsigned &gathered)
{
    const int c = __popc(M);
    if (c > 16)
        return warp_serve_d2<C5, 1>(L, M, lane, p, px, py, pt, s, best, gathered);
    if (c > 8)
        return warp_serve_d2<C5, 2>(L, M, lane, p, px, py, pt, s, best, gathered);
    if (c > 4)
        return warp_serve_d2<C5, 4>(L, M, lane, p, px, py, pt, s, best, gathered);
    return warp_serve_d2<C5, 8>(L, M, lane, p, px, py, pt, s, best, gathered);
}

// The FP16 screen (group_screen) of the pending candidates of M, the same way
// (the owner's magnitude bound D too).
template <bool C5, int G>
__device__ __forceinline__ bool warp_serve_screen(const LevelView &L, unsigned M, int lane, int p, int px, int py,
                                                  int pt, int s, float best, float D, unsigned &gathered_h)
{
    const unsigned FULL = 0xffffffffu;
    const int c = __popc(M);
    const int j = lane / G;
    const int o = j < c ? (int)__fns(M, 0, j + 1) : lane;
    const int op = __shfl_sync(FULL, p, o), opx = __shfl_sync(FULL, px, o), opy = __shfl_sync(FULL, py, o),
              opt = __shfl_sync(FULL, pt, o), os = __shfl_sync(FULL, s, o);
    const float ob = __shfl_sync(FULL, best, o), oD = __shfl_sync(FULL, D, o);
    int pass = 0;
    if (j < c)
        pass = group_screen<C5, G>(LevelView(L), op, opx, opy, opt, os, ob, oD, lane & (G - 1), group_mask<G>(),
                                   gathered_h);
    const int r = __popc(M & ((1u << lane) - 1u));
    return __shfl_sync(FULL, pass, (r * G) & 31) != 0;
}

template <bool C5>
__device__ __forceinline__ bool warp_screen(const LevelView &L, unsigned M, int lane, int p, int px, int py,
                                            int pt, int s, float best, float D, unsigned &gathered_h)
{
    const int c = __popc(M);
    if (c > 16)
        return warp_serve_screen<C5, 1>(L, M, lane, p, px, py, pt, s, best, D, gathered_h);
    if (c > 8)
        return warp_serve_screen<C5, 2>(L, M, lane, p, px, py, pt, s, best, D, gathered_h);
    if (c > 4)
        return warp_serve_screen<C5, 4>(L, M, lane, p, px, py, pt, s, best, D, gathered_h);
    return warp_serve_screen<C5, 8>(L, M, lane, p, px, py, pt, s, best, D, gathered_h);
}

// One round of the propagation candidates of a warp: the pending (target,
// candidate j) pairs are numbered candidate by candidate, lanes in order
// (Mj: the lanes whose candidate j is pending; n0, n1: the counts of M0,
// M1; c: all of them), and group g of G lanes serves pair base + g with its
// owner's target, source s[j] and bound. Each owner receives the distances
// of its pairs served in this round into out[j].
template <bool C5, int G>
__device__ __forceinline__ void multi_round(const LevelView &L, unsigned M0, unsigned M1, unsigned M2, int n0,
                                            int n1, int c, int base, int lane, int p, int px, int py, int pt,
                                            int s0, int s1, int s2, float best, float (&out)[3],
                                            unsigned &gathered)
{
    const unsigned FULL = 0xffffffffu;
    const int q = base + lane / G;
    int which = 0, o = lane;
    if (q < c) {
        if (q < n0) {
            o = (int)__fns(M0, 0, q + 1);
        } else if (q < n0 + n1) {
            which = 1;
            o = (int)__fns(M1, 0, q - n0 + 1);
        } else {
            which = 2;
            o = (int)__fns(M2, 0, q - n0 - n1 + 1);
        }
    }
    const int op = __shfl_sync(FULL, p, o), opx = __shfl_sync(FULL, px, o), opy = __shfl_sync(FULL, py, o),
              opt = __shfl_sync(FULL, pt, o);
    const int os0 = __shfl_sync(FULL, s0, o), os1 = __shfl_sync(FULL, s1, o), os2 = __shfl_sync(FULL, s2, o);
    const float ob = __shfl_sync(FULL, best, o);
    float dd = __int_as_float(0x7f800000);
    if (q < c)
        dd = group_d2<C5, G, false>(LevelView(L), op, opx, opy, opt, which == 0 ? os0 : which == 1 ? os1 : os2,
                                    nullptr, ob,
                                    lane & (G - 1), group_mask<G>(), gathered);
    const unsigned lt = (1u << lane) - 1u;
    const int cap = 32 / G;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const unsigned Mj = j == 0 ? M0 : j == 1 ? M1 : M2;
        const int qj = (j == 0 ? 0 : j == 1 ? n0 : n0 + n1) + __popc(Mj & lt);
        const bool here = ((Mj >> lane) & 1u) && qj >= base && qj < base + cap;
        const float r = __shfl_sync(FULL, dd, here ? ((qj - base) * G) & 31 : lane);
        if (here)
            out[j] = r;
    }
}

// The distances of all pending propagation candidates of a warp, bounded by
// each target's distance before them: one round when at most 32 are
// pending (G lanes each, the most that still serve them all, up to 8),
// else rounds of 32 with one lane each.
template <bool C5>
__device__ __forceinline__ void warp_d2_multi(const LevelView &L, unsigned M0, unsigned M1, unsigned M2, int lane,
                                              int p, int px, int py, int pt, int s0, int s1, int s2, float best,
                                              float (&out)[3], unsigned &gathered)
{
    const int n0 = __popc(M0), n1 = __popc(M1), c = n0 + n1 + __popc(M2);
    if (c > 16) {
        for (int base = 0; base < c; base += 32)
            multi_round<C5, 1>(L, M0, M1, M2, n0, n1, c, base, lane, p, px, py, pt, s0, s1, s2, best, out,
                                      gathered);
    } else if (c > 8) {
        multi_round<C5, 2>(L, M0, M1, M2, n0, n1, c, 0, lane, p, px, py, pt, s0, s1, s2, best, out,
                                  gathered);
    } else if (c > 4) {
        multi_round<C5, 4>(L, M0, M1, M2, n0, n1, c, 0, lane, p, px, py, pt, s0, s1, s2, best, out,
                                  gathered);
    } else {
        multi_round<C5, 8>(L, M0, M1, M2, n0, n1, c, 0, lane, p, px, py, pt, s0, s1, s2, best, out,
                                  gathered);
    }
}

// ann_one for the targets of a warp with warp-shared lanes: the whole warp
// calls it, and lane l owns target i of the clip a describes when active (all
// lanes of a warp belong to one clip; a batch pads every clip's range to whole
// warps). Without STAGES the propagation candidates of all its targets are
// gathered together and decided in order (see below); with STAGES they are
// judged one neighbour at a time, each bounded by the running best. Then each
// random-search stage offers at most one candidate per target, judged against
// the running best as in ann_one. The warp leaves a stage loop together, when
// no lane has a stage left. The two forms take the same decisions. Measured
// on GB300: the single clip (320x240x60) 18.5 ms per inpainting merged
// against 19.9 one by one; the 48-clip batch 1,487 ms merged against 1,403
// one by one (the merged round gathers 2% fewer voxels but its step launches
// take 10% longer there), so the single-clip kernel merges and the batch
// kernel does not.
template <bool C5, bool F16, bool STAGES>
__device__ __forceinline__ void ann_one_warp(const AnnArgs &a, bool active, int i, int k, int span, bool do_random,
                                             StepCount &n)
{
    const LevelView L = a.L;   // a register copy (the batch kernels read a from global memory)
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    // with FP16 storage, a level whose view carries no FP16 copy is searched
    // without screening (warp-uniform: a warp holds targets of one clip)
    const bool screen = F16 && L.h4 != nullptr;
    const float D = (screen && active) ? screen_d2bound(L) : 0.0f;
    const float INF = __int_as_float(0x7f800000);
    int p = 0, px = 0, py = 0, pt = 0;
    Shift cur;
    cur.dx = cur.dy = cur.dt = 0;
    float d = INF;
    Shift cn[3];
    int sn[3] = {-1, -1, -1};
    bool stale[3] = {false, false, false};
    if (active) {
        p = a.targets[i];
        decode(p, L.W, L.HW, px, py, pt);
        cur = a.phi_in[p];
        d = a.d_in[p];
        const int sg = (k & 1) ? 1 : -1;
        const bool in0 = inside(L, px + sg, py, pt), in1 = inside(L, px, py + sg, pt),
                   in2 = inside(L, px, py, pt + sg);
        const int r0 = in0 ? p + sg : p, r1 = in1 ? p + sg * L.W : p, r2 = in2 ? p + sg * L.HW : p;
        const bool t0 = in0 && (a.tmask[r0] & a.tbit), t1 = in1 && (a.tmask[r1] & a.tbit),
                   t2 = in2 && (a.tmask[r2] & a.tbit);
        cn[0] = a.phi_in[r0];
        cn[1] = a.phi_in[r1];
        cn[2] = a.phi_in[r2];
        sn[0] = t0 ? source_of(L, px, py, pt, cn[0].dx, cn[0].dy, cn[0].dt) : -1;
        sn[1] = t1 ? source_of(L, px, py, pt, cn[1].dx, cn[1].dy, cn[1].dt) : -1;
        sn[2] = t2 ? source_of(L, px, py, pt, cn[2].dx, cn[2].dy, cn[2].dt) : -1;
        // the change-flag rule of ann_one
        const unsigned span_mask = a.chg_in != nullptr && span > 0 ? (1u << span) - 1u : 0u;
        stale[0] = span_mask && t0 && (a.chg_in[r0] & span_mask) == 0;
        stale[1] = span_mask && t1 && (a.chg_in[r1] & span_mask) == 0;
        stale[2] = span_mask && t2 && (a.chg_in[r2] & span_mask) == 0;
    }
    Rejected rej;
    const Shift start = cur;
    if (STAGES) {
        // every candidate judged one stage at a time: the three neighbours,
        // then the random search, each bounded by the running best
#pragma unroll 1
        for (int stage = 0;; ++stage) {
            int s = -1, cdx = 0, cdy = 0, cdt = 0;
            bool skip = false;
            // does this lane's target have a candidate at this stage
            bool mine = active;
            int ri = 0, sh = 0;
            if (stage >= 3 && active) {
                ri = stage - 3;
                sh = a.rs_mode ? a.rho_log2 * ri : a.rho_log2 * k;
                mine = do_random && (a.rs_mode ? (ri < 31 && sh <= 30 && (a.rmax >> sh) >= 1) : ri == 0);
            }
            if (!__any_sync(FULL, mine))
                break;
            if (stage < 3) {
                // (a register array indexed by a loop variable would spill: select)
                const Shift c = stage == 0 ? cn[0] : (stage == 1 ? cn[1] : cn[2]);
                s = stage == 0 ? sn[0] : (stage == 1 ? sn[1] : sn[2]);
                skip = stage == 0 ? stale[0] : (stage == 1 ? stale[1] : stale[2]);
                cdx = c.dx;
                cdy = c.dy;
                cdt = c.dt;
            } else if (mine) {
                const uint4 w = philox4x32_10(make_uint4((uint32_t)p, a.tag | (uint32_t)k, a.clip,
                                                         a.rs_mode ? (uint32_t)ri : 0u),
                                              a.key0, a.key1);
                cdx = cur.dx + random_offset(w.x, a.rmax, sh + 24);
                cdy = cur.dy + random_offset(w.y, a.rmax, sh + 24);
                cdt = cur.dt + random_offset(w.z, a.rmax, sh + 24);
                s = source_of(L, px, py, pt, cdx, cdy, cdt);
            }
            bool need = false;
            unsigned long long key = 0;
            if (active && s >= 0) {
                ++n.evals;
                if (!skip) {
                    key = shift_key(cdx, cdy, cdt);
                    need = !(key == shift_key(cur.dx, cur.dy, cur.dt) || rej.has(key));
                }
            }
            if (screen && stage >= 3) {
                const unsigned M = __ballot_sync(FULL, need);
                if (M) {
                    const bool pass = warp_screen<C5>(L, M, lane, p, px, py, pt, s, d, D, n.gathered_h);
                    if (need) {
                        ++n.screened;
                        if (pass) {
                            ++n.passed;
                        } else {
                            rej.add(key);
                            need = false;
                        }
                    }
                }
            }
            const unsigned M = __ballot_sync(FULL, need);
            if (M) {
                const float dd = warp_d2<C5>(L, M, lane, p, px, py, pt, s, d, n.gathered);
                if (need) {
                    if (dd < d) {
                        d = dd;
                        cur.dx = (short)cdx;
                        cur.dy = (short)cdy;
                        cur.dt = (short)cdt;
                    } else {
                        rej.add(key);
                    }
                }
            }
        }
    } else {
        // Propagation: the three neighbours' candidates are gathered
        // together, each bounded by the distance the target had before them, and
        // then decided in order against the running best. A gather the bound
        // stopped is at or above every later best, and a completed one has the
        // exact distance, so the decisions are those of judging them one by one.
        // A candidate equal to the current shift, or to an earlier candidate of
        // the same target that is gathered, is decided by that one. (320x240x60:
        // 18.5 against 19.9 ms per inpainting; the 8-clip batch, its clips'
        // ranges padded to whole warps: 252.9 against 263.8 ms per batch with
        // the candidates judged one neighbour at a time in warps that mix
        // clips.)
        {
            bool need[3] = {false, false, false};
            unsigned long long key[3] = {0ull, 0ull, 0ull};
            if (active) {
                const unsigned long long k_cur = shift_key(cur.dx, cur.dy, cur.dt);
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    if (sn[j] < 0)
                        continue;
                    ++n.evals;
                    if (stale[j])
                        continue;
                    key[j] = shift_key(cn[j].dx, cn[j].dy, cn[j].dt);
                    bool nj = key[j] != k_cur;
#pragma unroll
                    for (int i = 0; i < j; ++i)
                        nj = nj && !(need[i] && key[i] == key[j]);
                    need[j] = nj;
                }
            }
            const unsigned M0 = __ballot_sync(FULL, need[0]), M1 = __ballot_sync(FULL, need[1]),
                           M2 = __ballot_sync(FULL, need[2]);
            if (M0 | M1 | M2) {
                float dist[3] = {INF, INF, INF};
                warp_d2_multi<C5>(L, M0, M1, M2, lane, p, px, py, pt, sn[0], sn[1], sn[2], d, dist, n.gathered);
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    if (!need[j])
                        continue;
                    if (dist[j] < d) {
                        d = dist[j];
                        cur = cn[j];
                    } else {
                        rej.add(key[j]);
                    }
                }
            }
        }
        // random search
#pragma unroll 1
        for (int stage = 3;; ++stage) {
            int s = -1, cdx = 0, cdy = 0, cdt = 0;
            // does this lane's target have a candidate at this stage
            bool mine = false;
            int ri = 0, sh = 0;
            if (active) {
                ri = stage - 3;
                sh = a.rs_mode ? a.rho_log2 * ri : a.rho_log2 * k;
                mine = do_random && (a.rs_mode ? (ri < 31 && sh <= 30 && (a.rmax >> sh) >= 1) : ri == 0);
            }
            if (!__any_sync(FULL, mine))
                break;
            if (mine) {
                const uint4 w = philox4x32_10(make_uint4((uint32_t)p, a.tag | (uint32_t)k, a.clip,
                                                         a.rs_mode ? (uint32_t)ri : 0u),
                                              a.key0, a.key1);
                cdx = cur.dx + random_offset(w.x, a.rmax, sh + 24);
                cdy = cur.dy + random_offset(w.y, a.rmax, sh + 24);
                cdt = cur.dt + random_offset(w.z, a.rmax, sh + 24);
                s = source_of(L, px, py, pt, cdx, cdy, cdt);
            }
            bool need = false;
            unsigned long long key = 0;
            if (active && s >= 0) {
                ++n.evals;
                key = shift_key(cdx, cdy, cdt);
                need = !(key == shift_key(cur.dx, cur.dy, cur.dt) || rej.has(key));
            }
            if (screen) {
                const unsigned M = __ballot_sync(FULL, need);
                if (M) {
                    const bool pass = warp_screen<C5>(L, M, lane, p, px, py, pt, s, d, D, n.gathered_h);
                    if (need) {
                        ++n.screened;
                        if (pass) {
                            ++n.passed;
                        } else {
                            rej.add(key);
                            need = false;
                        }
                    }
                }
            }
            const unsigned M = __ballot_sync(FULL, need);
            if (M) {
                const float dd = warp_d2<C5>(L, M, lane, p, px, py, pt, s, d, n.gathered);
                if (need) {
                    if (dd < d) {
                        d = dd;
                        cur.dx = (short)cdx;
                        cur.dy = (short)cdy;
                        cur.dt = (short)cdt;
                    } else {
                        rej.add(key);
                    }
                }
            }
        }
    }
    if (active) {
        a.phi_out[p] = cur;
        a.d_out[p] = d;
        if (a.chg_out) {
            const bool changed = cur.dx != start.dx || cur.dy != start.dy || cur.dt != start.dt;
            a.chg_out[p] = (uint8_t)((changed ? 1u : 0u) | ((unsigned)a.chg_in[p] << 1));
        }
    }
}

// Adds a launch's per-lane counts to the counters ctr[0..4] = evaluations,
// FP32 voxels, FP16 voxels, screened, passed (evaluations and candidate
// counts once per group).
template <bool F16>
__device__ __forceinline__ void flush_counts(unsigned long long *ev, unsigned long long *ga,
                                             unsigned long long *scr, const StepCount &n, int sub)
{
    count_evals(ev, sub == 0 ? n.evals : 0u);
    count_evals(ga, n.gathered);
    if (F16) {
        count_evals(scr, n.gathered_h);
        count_evals(scr + 1, sub == 0 ? n.screened : 0u);
        count_evals(scr + 2, sub == 0 ? n.passed : 0u);
    }
}

template <bool C5, int G, bool PARTIAL, bool F16>
__global__ void __launch_bounds__(STEP_BLOCK, step_min_blocks<G, PARTIAL>() * (256 / STEP_BLOCK))
    k_ann_step(const AnnArgs a)
{
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gt / G;
    const int sub = gt & (G - 1);
    const unsigned gmask = group_mask<G>();
    StepCount n;
    if (i < a.nT)
        ann_one<C5, G, PARTIAL, F16>(a, i, a.k, a.chg_span, a.do_random != 0, sub, gmask, n);
    flush_counts<F16>(a.evals, a.gathered, a.screen, n, sub);
}

// One target per lane, candidates' gathers shared by the warp (lanes = 32).
template <bool C5, bool F16>
__global__ void __launch_bounds__(STEP_BLOCK, 2 * (256 / STEP_BLOCK)) k_ann_step_warp(const AnnArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    StepCount n;
    ann_one_warp<C5, F16, false>(a, i < a.nT, i, a.k, a.chg_span, a.do_random != 0, n);
    flush_counts<F16>(a.evals, a.gathered, a.screen, n, 0);
}

// Batch form: the targets of n clips in one persistent launch. Clip c owns
// the global target indices [prefix[c], prefix[c+1]) and is described by
// clips[c]; every clip runs sweep w (BatchSweep: iteration k, sweep index,
// change-flag span, random search or propagation only). Sweep index s reads
// shift buffer s & 1 (clips[c].odd for even s) and writes the other. A
// grid-stride loop over groups keeps the grid at the resident size whatever
// the batch holds. ctr: evaluations, FP32 voxels, FP16 voxels, screened,
// passed.
template <bool C5, int G, bool F16>
__global__ void __launch_bounds__(STEP_BLOCK, step_min_blocks<G, false>() * (256 / STEP_BLOCK))
    k_ann_step_batch(const BatchClip *__restrict__ clips, const int *__restrict__ prefix, int n, BatchSweep w,
                     unsigned long long *ctr)
{
    const int total = __ldg(prefix + n);
    const int sub = (blockIdx.x * blockDim.x + threadIdx.x) & (G - 1);
    const unsigned gmask = group_mask<G>();
    const int stride = gridDim.x * blockDim.x / G;
    StepCount cnt;
    for (int g = (blockIdx.x * blockDim.x + threadIdx.x) / G; g < total; g += stride) {
        const int c = find_segment(prefix, n, g);
        const AnnArgs &a = (w.sweep & 1) ? clips[c].even : clips[c].odd;
        const int i = g - __ldg(prefix + c);
        if (i < a.nT)   // a clip's range is padded to whole warps
            ann_one<C5, G, false, F16>(a, i, w.k, w.span, w.do_random != 0, sub, gmask, cnt);
    }
    flush_counts<F16>(ctr, ctr + 1, ctr + 2, cnt, sub);
}

// Batch form of the warp-shared step: warp v of the grid-stride loop takes
// the global targets [32 v, 32 v + 32). Every clip's range starts on a whole
// warp (the host pads the prefix sums to multiples of 32), so a warp holds
// targets of one clip only; its candidates are judged one stage at a time.
template <bool C5, bool F16>
__global__ void __launch_bounds__(STEP_BLOCK, 2 * (256 / STEP_BLOCK))
    k_ann_step_batch_warp(const BatchClip *__restrict__ clips, const int *__restrict__ prefix, int n, BatchSweep w,
                          unsigned long long *ctr)
{
    const int total = __ldg(prefix + n);
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x / 32);
    StepCount cnt;
    for (int v = (blockIdx.x * blockDim.x + threadIdx.x) / 32; v * 32 < total; v += warps) {
        const int c = find_segment(prefix, n, v * 32);
        const AnnArgs &a = (w.sweep & 1) ? clips[c].even : clips[c].odd;
        const int i = v * 32 - __ldg(prefix + c) + lane;
        ann_one_warp<C5, F16, true>(a, i < a.nT, i < a.nT ? i : 0, w.k, w.span, w.do_random != 0, cnt);
    }
    flush_counts<F16>(ctr, ctr + 1, ctr + 2, cnt, 0);
}

template <bool C5, int G, bool PARTIAL, bool F16>
void launch_ann_step_g(const AnnArgs &a, cudaStream_t st)
{
    k_ann_step<C5, G, PARTIAL, F16><<<blocks_for((long long)a.nT * G, STEP_BLOCK), STEP_BLOCK, 0, st>>>(a);
}

// The single-clip step with storage F16 (launch counted by the caller).
template <bool F16>
void launch_ann_step_impl(const AnnArgs &a, bool c5, cudaStream_t st)
{
    if (!F16 && a.excl) {
        if (c5)
            launch_ann_step_g<true, 8, true, false>(a, st);
        else
            launch_ann_step_g<false, 8, true, false>(a, st);
        return;
    }
    if (a.lanes == 32) {
        const int grid = blocks_for(a.nT, STEP_BLOCK);
        if (c5)
            k_ann_step_warp<true, F16><<<grid, STEP_BLOCK, 0, st>>>(a);
        else
            k_ann_step_warp<false, F16><<<grid, STEP_BLOCK, 0, st>>>(a);
        return;
    }
    switch ((a.lanes > 0 ? a.lanes : pick_group(a.nT)) * 2 + (c5 ? 1 : 0)) {
    case 2: launch_ann_step_g<false, 1, false, F16>(a, st); break;
    case 3: launch_ann_step_g<true, 1, false, F16>(a, st); break;
    case 4: launch_ann_step_g<false, 2, false, F16>(a, st); break;
    case 5: launch_ann_step_g<true, 2, false, F16>(a, st); break;
    case 8: launch_ann_step_g<false, 4, false, F16>(a, st); break;
    case 9: launch_ann_step_g<true, 4, false, F16>(a, st); break;
    case 16: launch_ann_step_g<false, 8, false, F16>(a, st); break;
    default: launch_ann_step_g<true, 8, false, F16>(a, st); break;
    }
}

template <bool C5, int G, bool F16>
void launch_ann_step_batch_g(const BatchClip *clips, const int *tprefix, int n, int total, BatchSweep k,
                             unsigned long long *ctr, cudaStream_t st)
{
    k_ann_step_batch<C5, G, F16><<<persistent_grid((long long)total * G,
                                                   step_min_blocks<G, false>() * (256 / STEP_BLOCK), STEP_BLOCK),
                                   STEP_BLOCK, 0, st>>>(clips, tprefix, n, k, ctr);
}

template <bool F16>
void launch_ann_step_batch_impl(const BatchClip *clips, const int *tprefix, int n, int total, BatchSweep k, bool c5,
                                unsigned long long *ctr, int lanes, cudaStream_t st)
{
    if (lanes == 32) {
        const int grid = persistent_grid(total, 2 * (256 / STEP_BLOCK), STEP_BLOCK);
        if (c5)
            k_ann_step_batch_warp<true, F16><<<grid, STEP_BLOCK, 0, st>>>(clips, tprefix, n, k, ctr);
        else
            k_ann_step_batch_warp<false, F16><<<grid, STEP_BLOCK, 0, st>>>(clips, tprefix, n, k, ctr);
        return;
    }
    switch ((lanes > 0 ? lanes : pick_group(total)) * 2 + (c5 ? 1 : 0)) {
    case 2: launch_ann_step_batch_g<false, 1, F16>(clips, tprefix, n, total, k, ctr, st); break;
    case 3: launch_ann_step_batch_g<true, 1, F16>(clips, tprefix, n, total, k, ctr, st); break;
    case 4: launch_ann_step_batch_g<false, 2, F16>(clips, tprefix, n, total, k, ctr, st); break;
    case 5: launch_ann_step_batch_g<true, 2, F16>(clips, tprefix, n, total, k, ctr, st); break;
    case 8: launch_ann_step_batch_g<false, 4, F16>(clips, tprefix, n, total, k, ctr, st); break;
    case 9: launch_ann_step_batch_g<true, 4, F16>(clips, tprefix, n, total, k, ctr, st); break;
    case 16: launch_ann_step_batch_g<false, 8, F16>(clips, tprefix, n, total, k, ctr, st); break;
    default: launch_ann_step_batch_g<true, 8, F16>(clips, tprefix, n, total, k, ctr, st); break;
    }
}

}  // namespace vi
