// vi_launch.h -- host-side launchers of the library's kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "vi_device.cuh"

namespace vi {
// Kernel launches issued by this library in this process (all contexts).
extern std::atomic<unsigned long long> g_launch_count;
}  // namespace vi
#define VI_COUNT_LAUNCH() (::vi::g_launch_count.fetch_add(1, std::memory_order_relaxed))

namespace vi {

// ---- pyramid and sets (vi_pyramid.cu) --------------------------------------
// Grey-level derivatives of the level-0 video: g = (|I_x|, |I_y|), valid bits
// (1: I_x known, 2: I_y known) -- Eq. 7.
void launch_gradients(const float *rgb, const uint8_t *hole, int W, int H, int T, float2 *g,
                      uint8_t *valid, cudaStream_t st);
// Box mean of g over the square nu of side `side` (Eq. 7) -> T0 = (T_x, T_y).
void launch_box_mean(const float2 *g, const uint8_t *valid, int W, int H, int T, int side,
                     float2 *tmp_sum, uint16_t *tmp_cnt, float2 *T0, cudaStream_t st);
// Level-0 channels from the input video and T0 (occluded voxels zeroed).
void launch_level0_channels(const float *rgb, const uint8_t *hole, const float2 *T0,
                            float sqrt_lambda, bool c5, LevelView L, cudaStream_t st);
// Coarse level from the finer one: 2x2 mean of known children, OR of the
// occlusion, texture features subsampled from T0 (Eq. 8).
// tsub: the temporal subsampling option (coarse frames = ceil(fine / 2)).
void launch_downsample(LevelView fine, LevelView coarse, int level, const float2 *T0, int W0,
                       int H0, float sqrt_lambda, bool c5, bool tsub, cudaStream_t st);
// code = H | H~ | D~ of a level from its occlusion bits (3 separable dilations).
void launch_codes(LevelView L, uint8_t *tmp_a, uint8_t *tmp_b, cudaStream_t st);
// out[t] = (x0, x1, y0, y1) of the occluded pixels of frame t ((W, -1, H, -1): none).
void launch_mask_extents(const uint8_t *mask, int W, int H, int T, int4 *out, cudaStream_t st);
// Raster-ordered compaction of {v : (flags[v] & bits) != 0} into list.
// block_counts needs compact_blocks(V) + 1 ints; *count_dev receives the size.
int compact_blocks(int V);
// Three lists at once: block_counts needs 3 * (compact_blocks(V) + 1) ints,
// which the write pass reads again; count_dev[0..2] receive the sizes.
void launch_compact3_count(const uint8_t *flags, uchar3 bits, int V, int *block_counts, int *count_dev,
                           cudaStream_t st);
void launch_compact3_write(const uint8_t *flags, uchar3 bits, int V, const int *block_counts, int *l0, int *l1,
                           int *l2, cudaStream_t st);
void launch_compact(const uint8_t *flags, uint8_t bits, int V, int *block_counts, int *list,
                    int *count_dev, cudaStream_t st);

// ---- search (vi_search.cu) ----------------------------------------------------
struct AnnArgs {
    LevelView L;
    const int *targets;
    int nT;
    const Shift *phi_in;
    const float *d_in;
    Shift *phi_out;
    float *d_out;
    const uint8_t *tmask;  // neighbour r is a target iff tmask[r] & tbit
    uint8_t tbit;
    const uint8_t *excl;   // partial distance (Eq. 11) when non-null
    int k;                 // PatchMatch iteration 1..n_pm
    int rmax;
    int rho_log2;          // rho = 2^-rho_log2
    uint32_t key0, key1, tag, clip;
    unsigned long long *evals;     // candidate evaluations (valid candidates)
    unsigned long long *gathered;  // FP32 source voxels actually read
    unsigned long long *screen;    // FP16 storage: FP16 voxels read, screened, passed (3 counters)
    int lanes;                     // lanes per target (1, 2, 4, 8); 0: by target count
    int rs_mode;                   // 0: one random candidate at radius rmax rho^k (Eq. 3);
                                   // 1: one at every radius rmax rho^i >= 1, i = 0, 1, ...
    int do_random;                 // 0: propagation only (a sub-sweep before the last)
    // Change history: chg_in[r] bit i = r's shift changed in the sweep i + 1
    // sweeps back; chg_out receives the history after this sweep. chg_span >
    // 0 (single-clip launches; the batch step derives it from k): the sweeps
    // since this target last judged the same neighbours in the same
    // direction; a neighbour unchanged over all of them offers no new
    // candidate. nullptr / 0: no history.
    const uint8_t *chg_in;
    uint8_t *chg_out;
    int chg_span;
};
// FP16 screening when a.L.h4 is set (full distance only; the partial
// distance of Eq. 11 always runs on the FP32 channels).
void launch_ann_step(const AnnArgs &a, bool c5, cudaStream_t st);
void launch_ann_step_f16(const AnnArgs &a, bool c5, cudaStream_t st);
// d_out[p] = distance of target p to p + phi[p] (in place allowed).
void launch_rescore(LevelView L, const int *targets, int nT, const Shift *phi, float *d_out,
                    const uint8_t *excl, bool c5, unsigned long long *evals, cudaStream_t st,
                    int lanes = 0);
void launch_copy_targets(const int *targets, int nT, const Shift *phi_src, const float *d_src,
                         Shift *phi_dst, float *d_dst, cudaStream_t st);
void launch_init_nnf(LevelView L, const int *targets, int nT, const int *sources, int nS,
                     Shift *phi, uint32_t key0, uint32_t key1, uint32_t tag, uint32_t clip,
                     cudaStream_t st);
void launch_upsample_nnf(LevelView coarse, const Shift *phi_c, LevelView fine, bool tsub,
                         const int *targets_f, int nT, const int *sources_f, int nS, Shift *phi_f, uint32_t key0,
                         uint32_t key1, uint32_t tag, uint32_t clip, cudaStream_t st);
void launch_provisional_fill(LevelView coarse, LevelView fine, const int *holes_f, int nH,
                             bool c5, bool tsub, cudaStream_t st);
void launch_patch_dist(LevelView L, const int *pairs, int n, float *out, bool c5, cudaStream_t st);
void launch_patch_dist_partial(LevelView L, const int *pairs, int n, const uint8_t *excl, float *out, bool c5,
                               cudaStream_t st);

// ---- reconstruction (vi_vote.cu) -----------------------------------------------
struct VoteArgs {
    LevelView L;
    const int *list;       // voxels to reconstruct
    int n;
    const Shift *phi;
    const float *d2;
    const uint8_t *allowed;  // q contributes iff allowed[q] & abit; null: every in-video q
    uint8_t abit;
    int weighted;
    uint8_t *hp;           // onion peel: cleared for filled voxels (nullable)
    float *partials;       // per-block sum of |change| over the colour channels
};
void launch_vote(const VoteArgs &a, bool c5, cudaStream_t st);
// out[0] = sum of partials[0..n) in a fixed order, in two stages; chunks
// holds sum_chunks(n) doubles of scratch.
int sum_chunks(int n);
void launch_sum_partials(const float *partials, int n, double *chunks, double *out, cudaStream_t st);
// out[i] = sum of vals[starts[i] .. starts[i+1]) in the same fixed order;
// cprefix[i] = sum of sum_chunks over the segments before i (nseg + 1
// entries, total_chunks = cprefix[nseg]); chunks holds total_chunks doubles.
// starts and cprefix in device memory.
void launch_segment_sums(const float *vals, const int *starts, const int *cprefix, int nseg, int total_chunks,
                         double *chunks, double *out, cudaStream_t st);
void launch_final(LevelView L, const int *holes, int nH, const Shift *phi, const float *d2,
                  bool c5, cudaStream_t st);
int energy_blocks(int n);
void launch_energy(LevelView L, const int *targets, int nT, const Shift *phi, bool c5,
                   double *partials2, cudaStream_t st);
void launch_sum_partials2(const double *partials2, int n, double *out2, cudaStream_t st);
// ---- batches of clips (one launch for the current level of every clip) -----
// odd: arguments of the odd PatchMatch iterations (read buffer 0, write 1);
// even: the even ones (read 1, write 0); vote: the clip's reconstruction,
// whose partials point at the clip's slice of the batch's per-voxel array;
// d0: buffer 0 of the distances (written by the batch rescore).
struct BatchClip {
    AnnArgs odd;
    AnnArgs even;
    VoteArgs vote;
    float *d0;
};
// One Jacobi sweep of a batch round: PatchMatch iteration k (1..n_pm; the
// scan direction and the Philox counter), sweep index (0-based over the
// round's n_pm * sub_sweeps sweeps: sweep s reads shift buffer s & 1),
// change-flag span (as AnnArgs::chg_span), and whether the sweep ends with
// the random search (the last sub-sweep of an iteration) or only propagates.
struct BatchSweep {
    int k;
    int sweep;
    int span;
    int do_random;
};
// clips[c] owns targets [tprefix[c], tprefix[c+1]) / holes [hprefix[c],
// hprefix[c+1]); prefixes in device memory (n + 1 entries); totals on the host.
// ctr: evaluations, FP32 voxels read, FP16 voxels read, screened, passed.
void launch_ann_step_batch(const BatchClip *clips, const int *tprefix, int n, int total_targets, BatchSweep w,
                           bool c5, bool f16, unsigned long long *ctr, int lanes, cudaStream_t st);
void launch_ann_step_batch_f16(const BatchClip *clips, const int *tprefix, int n, int total_targets, BatchSweep w,
                               bool c5, unsigned long long *ctr, int lanes, cudaStream_t st);
void launch_rescore_batch(const BatchClip *clips, const int *tprefix, int n, int total_targets, bool c5,
                          unsigned long long *evals, int lanes, cudaStream_t st);
void launch_vote_batch(const BatchClip *clips, const int *hprefix, int n, int total_holes, bool c5,
                       cudaStream_t st);

// Onion peel sets on the coarsest level (Algorithm 3).
void launch_onion_layer(LevelView L, const uint8_t *hp, uint8_t *layer, cudaStream_t st);
void launch_onion_targets(LevelView L, const uint8_t *hp, const uint8_t *layer, uint8_t *ltgt,
                          cudaStream_t st);
void launch_count(const uint8_t *flags, int V, int *count_dev, cudaStream_t st);
// Packing helpers between the library layout and the ABI layout.
void launch_pack_rgb(LevelView L, float *rgb, cudaStream_t st);
// dst[0 .. n) = src[0 .. n) by a kernel; both must be device-accessible
// (device memory, or registered host memory through its device address).
void launch_copy_bytes(void *dst, const void *src, long long n, cudaStream_t st);
void launch_pack_voxels(LevelView L, const int *list, int n, float4 *buf4, float *buf1, bool unpack,
                        cudaStream_t st);
void launch_get_channels(LevelView L, float *out, int C, cudaStream_t st);
void launch_set_channels(LevelView L, const float *in, int C, cudaStream_t st);
// FP16 copies of channels c0..c3 of every voxel of a level (no-op for FP32
// storage).
void launch_shadow_all(LevelView L, cudaStream_t st);

}  // namespace vi

namespace vi {
// out[v] = (in[v] & bit) ? 1 : 0
void launch_extract_bit(const uint8_t *in, uint8_t bit, uint8_t *out, int V, cudaStream_t st);
// dst[v] = value for v < n
void launch_fill_f32(float *dst, float value, long long n, cudaStream_t st);
}  // namespace vi
