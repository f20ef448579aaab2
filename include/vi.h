/*
 * vi.h -- C ABI of the GB300 video-inpainting library.
 *
 * The library runs the per-pyramid-level hot path of the global patch-based
 * video inpainting method of Newson, Almansa, Fradet, Gousseau and Perez,
 * "Video Inpainting of Complex Scenes" (SIAM J. Imaging Sciences 7(4), 2014;
 * arXiv:1503.05528), Algorithm 4 (the affine realignment of Algorithm 2,
 * Sec. 3.4, is a separate set of calls around it): pyramids and texture
 * features (Sec. 3.3, Eq. 7, Eq. 8), shift-
 * map initialisation, onion-peel initialisation (Sec. 3.5, Algorithm 3),
 * spatio-temporal PatchMatch (Sec. 3.1, Algorithm 1, Eq. 2, Eq. 3, Eq. 7b),
 * weighted reconstruction (Sec. 3.2, Eq. 4, Eq. 5, Eq. 9), level transition
 * (Sec. 3.6), final best-patch reconstruction (Eq. 6), energy (Eq. 1) and the
 * stopping rule (Sec. 3.7). Every step runs in CUDA kernels for sm_103a.
 *
 * Conventions (all entry points):
 *  - Every call returns a vi_status; no exception crosses the ABI. On error
 *    vi_last_error() returns a message for the context.
 *  - Videos are float32 [T][H][W][3] (frame, row, column, RGB), values in [0, 1].
 *    Masks are uint8 [T][H][W], 1 = occluded (the set H of Sec. 2), 0 = known.
 *    Level l of the pyramid is ceil(W/2^l) x ceil(H/2^l) x T; level 0 is the
 *    input resolution (the paper's finest level).
 *  - Channels at a level are float32 [T][H][W][C]: R, G, B and, when texture
 *    features are on (C = 5), sqrt(lambda) T_x and sqrt(lambda) T_y, so that the
 *    distance of Eq. 7b is a plain sum of squares over C channels.
 *  - Shift maps are int32 [T][H][W][3] (dx, dy, dt): the correspondent of p is
 *    p + phi(p) (Sec. 2). Distances d2 are float32 [T][H][W], the squared patch
 *    distance d^2 of Eq. 2 / Eq. 7b. Both are meaningful on the target set H~
 *    (the dilated occlusion) only.
 *  - Pointers named *host* or taking ptr_is_device = 0 are host memory; with
 *    ptr_is_device = 1 they are device memory of the context's device. The
 *    caller owns every buffer it passes; the library copies what it keeps.
 *    The context owns all device state until vi_ctx_destroy.
 *  - The video of vi_upload (and the batch and server calls that take one) and
 *    the result of vi_fetch_result move between host and device by kernels
 *    that read or write the host buffer through its device address when it is
 *    registered with CUDA (cudaHostAlloc, cudaMallocHost, cudaHostRegister,
 *    or a framework's pinned memory), and by the copy engine otherwise; the
 *    results are the same either way.
 *  - Calls are ordered on the context's stream. Calls that return data to a
 *    host pointer synchronise that stream; the others are asynchronous unless
 *    stated otherwise.
 *  - A context is used by one thread at a time.
 *  - Limits: W, H, T <= 32767; W*H*T < 2^31; rho a power of two (1/2^m, m >= 1).
 */
#ifndef VI_H
#define VI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vi_ctx vi_ctx;

typedef enum {
    VI_OK = 0,
    VI_ERR_ARG = 1,        /* invalid argument (null pointer, size, level, config) */
    VI_ERR_OOM = 2,        /* device or host allocation failed */
    VI_ERR_CUDA = 3,       /* a CUDA call failed; vi_last_error() has the text */
    VI_ERR_TIMEOUT = 4,    /* a bounded wait gave up (reserved: no call waits on the device) */
    VI_ERR_NO_SOURCE = 5,  /* D~ is empty at some level: nothing to copy from */
    VI_ERR_STATE = 6,      /* call out of order (e.g. iterate before upload) */
    VI_ERR_NO_DEVICE = 7,  /* no CUDA device is available */
    VI_ERR_TOO_LARGE = 8   /* input larger than a fixed maximum: vi_energy_noalloc's
                              voxel count, a server's HBM budget */
} vi_status;

/* Parameters of the method (Sec. 3.7 gives the paper's values). */
typedef struct {
    float lambda;        /* texture-feature weight of Eq. 7b (paper: 50) */
    int n_pm;            /* PatchMatch iterations per ANN search, Algorithm 1 (10) */
    float rho;           /* random-search radius factor of Eq. 3 (0.5); 1/2^m only */
    int levels;          /* pyramid levels L >= 1 (0: choose by the rule of Sec. 3.6) */
    int max_outer;       /* cap on search/reconstruction iterations per level (20) */
    float stop;          /* threshold on e, the mean absolute colour change per
                            channel and voxel of H between iterations (0.1/255) */
    int weighted;        /* 1: weights of Eq. 5; 0: the unweighted mean (s = 1) */
    int use_texture;     /* 1: C = 5 channels (Sec. 3.3); 0: RGB only (C = 3) */
    int storage;         /* 0: FP32 channels. 1: FP32 channels plus an FP16 copy
                            of channels c0..c3 (8 B per voxel); at a level
                            whose FP32 channels are larger than the L2 cache
                            the PatchMatch step screens each random-search
                            candidate on that copy with a rigorous error bound
                            and computes the FP32 distance only when the
                            candidate could beat the current best (levels that
                            fit in L2 are searched as with storage 0). 2: the
                            same, screening at every level. Results are
                            identical to storage 0 in every mode (the paper
                            fixes no storage precision; this is a speed option
                            for clips larger than L2). */
    uint64_t seed;       /* Philox4x32-10 key (key words: low, high 32 bits) */
    uint32_t clip;       /* Philox counter word 2: distinguishes clips in a batch */
    int lanes_per_target; /* GPU lanes sharing one target in the search kernels:
                             0 = chosen per level from its size, or 1, 2, 4, 8;
                             32 = warp-shared: in the PatchMatch step each
                             lane owns a target and the lanes of a warp are
                             shared out among the candidates that need a
                             distance (the rescore then uses 1); never changes
                             a result, only the speed */
    int stream_priority; /* priority of the stream a context creates for itself
                            (vi_ctx_create with cuda_stream NULL): 0 default,
                            lower = scheduled first; clamped to the device's
                            range. Ignored when the caller passes a stream. */
    int rs_mode;         /* random search: 0 = Algorithm 1 / Eq. 3, one candidate
                            per PatchMatch iteration k at radius r_max rho^k;
                            1 = the original PatchMatch search, a candidate at
                            every radius r_max rho^i >= 1 (i = 0, 1, ...) per
                            k, each around the best shift so far (Sec. 3.1
                            discusses both) */
    int sub_sweeps;      /* propagation sweeps per PatchMatch iteration, the
                            last one followed by the random search; 1..16.
                            Default 2: a parallel (Jacobi) sweep spreads a
                            good shift one voxel where the paper's sequential
                            scan spreads it along the scan, and two sweeps per
                            iteration bring the energy of Eq. 1 within 2% of
                            the sequential search's (one, the paper's count,
                            leaves it about 4% above). A batch's clips share
                            the batch's value. */
    int time_subsample;  /* 0: pyramid levels keep every frame (Sec. 3.6); 1: the
                            option the paper uses once for long occlusions:
                            every level also halves the frames (2x2x2 means,
                            occlusion by OR, features sampled at (2^l x, 2^l y,
                            2^l t), shifts upsampled with dt doubled) */
    size_t mem_limit;    /* device bytes a context may hold at once (0: no
                            limit); an allocation beyond it fails with
                            VI_ERR_OOM as if the device were full, so the
                            failure paths can be exercised without
                            exhausting the GPU. vi_footprint_bytes is a
                            limit every run stays within. */
} vi_config;

/* Per-context counters. evals, step_*: since vi_ctx_create; outer and
 * onion_layers: since the last vi_upload. */
typedef struct {
    unsigned long long evals;          /* patch-distance evaluations (Eq. 2 / 7b / 11) */
    unsigned long long step_evals;     /* those made inside the PatchMatch step kernel */
    unsigned long long step_gathered;  /* source voxels the step kernel read: candidates
                                          equal to a shift already compared need none,
                                          and a gather stops once it cannot win */
    unsigned long long step_gathered_h; /* FP16 source voxels (8 B) the step kernel
                                          read (storage 1: candidate screening) */
    unsigned long long screened;       /* candidates screened on the FP16 copy */
    unsigned long long screen_passed;  /* of those, evaluated in FP32 */
    unsigned long long step_launches;  /* launches of the PatchMatch step kernel */
    double step_ms;                    /* device time of those launches (profiling on, see vi_profile) */
    unsigned long long step_timed;     /* launches included in step_ms */
    int outer[16];                     /* search/reconstruction iterations run per level */
    int onion_layers;                  /* layers peeled by the initialisation */
    int levels;                        /* levels of the current pyramid */
    unsigned long long launches;       /* kernels launched by the library in this
                                          process, all contexts together */
} vi_stats;

/* Fills cfg with the paper's parameters (Sec. 3.7), L = 0 (automatic), FP32,
 * texture features on, seed 1503. */
void vi_config_default(vi_config *cfg);

/* Creates a context on the current CUDA device. cuda_stream is a cudaStream_t
 * to order work on, or NULL for a stream the context creates and owns.
 * Errors: VI_ERR_ARG (bad config), VI_ERR_NO_DEVICE, VI_ERR_CUDA. */
vi_status vi_ctx_create(const vi_config *cfg, void *cuda_stream, vi_ctx **out);

/* Releases every device buffer and the owned stream. NULL is ignored. */
void vi_ctx_destroy(vi_ctx *ctx);

/* Message of the last failed call on ctx ("" if none). Valid until the next call. */
const char *vi_last_error(const vi_ctx *ctx);

/* The number of levels the rule of Sec. 3.6 picks for a mask: the smallest L
 * such that the largest per-frame occlusion extent (width or height of its
 * bounding box) divided by 2^(L-1) is at most 9, just under twice the patch
 * size of 5, keeping the coarsest frame side >= 16 px. Host-only. */
int vi_auto_levels(const uint8_t *mask_host, int W, int H, int T);

/* Device bytes a context will hold for a W x H x T clip with the given
 * number of occluded voxels (an upper bound used for admission; the lists
 * are bounded by the voxel count, so the bound does not depend on
 * hole_voxels at present). */
size_t vi_footprint_bytes(const vi_config *cfg, int W, int H, int T, long long hole_voxels);

/* Copies a video and its occlusion mask into the context and allocates the
 * pyramid. rgb: [T][H][W][3] float32; mask: [T][H][W] uint8. Values of rgb
 * under the mask are never read. Replaces any previous upload. From host
 * memory it returns once both buffers have been read (the context's stream
 * is synchronised), so the caller may reuse them at once; from device memory
 * it is stream-ordered like the other calls.
 * Errors: VI_ERR_ARG (sizes, null), VI_ERR_OOM, VI_ERR_CUDA. */
vi_status vi_upload(vi_ctx *ctx, const float *rgb, const uint8_t *mask, int W, int H, int T,
                    int ptr_is_device);

/* Algorithm 4, first three lines: the texture features at full resolution
 * (Eq. 7: mean over a square of side 2^(L-1) of the absolute central
 * differences of the grey level), the colour and occlusion pyramids (2x2
 * spatial means of known children, occlusion by OR, no temporal subsampling,
 * Sec. 3.6), the texture pyramid by subsampling (Eq. 8), and per level the
 * sets H~ and D~ of Sec. 2 with their raster-ordered voxel lists.
 * Errors: VI_ERR_STATE (no upload), VI_ERR_NO_SOURCE, VI_ERR_CUDA. */
vi_status vi_build_pyramid(vi_ctx *ctx);

/* Shift-map initialisation (Sec. 3.1; Algorithm 4, "phi^L <- Random"): every
 * voxel of H~ at the level takes a source drawn uniformly from D~.
 * Errors: VI_ERR_ARG (level), VI_ERR_STATE, VI_ERR_CUDA. */
vi_status vi_init_nnf(vi_ctx *ctx, int level);

/* Onion-peel initialisation at the coarsest level (Sec. 3.5, Algorithm 3):
 * layer by layer, the voxels of H' not kept by a 3x3x3 erosion are inpainted
 * from the patches that meet them and are centred outside H' (Eq. 10-12),
 * after an ANN search with the partial distance of Eq. 11.
 * Synchronises the stream once per layer. Errors: VI_ERR_STATE, VI_ERR_CUDA. */
vi_status vi_onion_peel(vi_ctx *ctx);

/* One layer of the onion-peel initialisation (Sec. 3.5, Algorithm 3,
 * Eq. 10-12) at the coarsest level, for checking the layers one by one on
 * injected state. With H' the voxels still to fill:
 *   dH' = H' minus its 3x3x3 erosion (voxels outside the video count as
 *         outside H');
 *   targets = voxels outside H' whose 5x5x5 patch meets dH';
 *   the ANN search of vi_ann on those targets with the partial distance of
 *   Eq. 11 (target voxels in H' left out, the sum divided by the count kept;
 *   +inf when none is), random draws tagged with `layer`;
 *   the vote of Eq. 12 of every voxel of dH' from the targets of its patch;
 *   a voxel of dH' that no target reaches stays in H'.
 * The channels, shift map and distances are the level's (vi_set_channels /
 * vi_set_nnf inject them). hprime_in: host uint8 [T][H][W] of the coarsest
 * level, nonzero = in H' (copied); NULL continues from the H' the previous
 * call left, or from the occluded set when no layer has run since the
 * pyramid was built. hprime_out (host, nullable) receives H' after the layer
 * (1 = still to fill); *n_left (nullable) its size. Synchronises. Errors:
 * VI_ERR_STATE (no pyramid), VI_ERR_ARG (layer outside [0, 65535]),
 * VI_ERR_CUDA. */
vi_status vi_onion_layer(vi_ctx *ctx, int layer, const uint8_t *hprime_in, uint8_t *hprime_out, int *n_left);

/* vi_build_pyramid + vi_init_nnf(levels-1) + vi_onion_peel. */
vi_status vi_prepare(vi_ctx *ctx);

/* Distances of every voxel of H~ at the level to its current correspondent
 * (d2 = d^2(W_p, W_{p+phi(p)}), Eq. 2 / 7b). */
vi_status vi_rescore(vi_ctx *ctx, int level);

/* One ANN search (Algorithm 1) at the level: vi_rescore, then n_pm
 * iterations of propagation and random search with the parallel (Jacobi)
 * schedule: in iteration k every target reads its neighbours' shifts as they
 * were when iteration k began; neighbours -e_x, -e_y, -e_t on even k, +e_x,
 * +e_y, +e_t on odd k; a candidate replaces the current shift only if it is
 * in D~ and strictly closer. The random candidate of iteration k is
 * p + phi(p) + floor(r_max rho^k delta) (Eq. 3), r_max the largest dimension
 * of the level and delta from Philox4x32-10 with counter (voxel index,
 * 0x2 << 28 | level << 24 | call << 8 | k, clip, 0). */
vi_status vi_ann(vi_ctx *ctx, int level, int call);

/* Reconstruction (Eq. 4, Eq. 5, and Eq. 9 for the texture channels) of every
 * occluded voxel at the level from the current shift map and distances:
 * sigma_p^2 is the 75th percentile (nearest rank) of the d2 of the patches
 * containing p. e_host (nullable) receives e = sum |u_new - u_old| over the
 * occluded voxels and the 3 colour channels / (3 |H|); a non-null e_host
 * synchronises the stream. */
vi_status vi_reconstruct(vi_ctx *ctx, int level, float *e_host);

/* The inner loop of Algorithm 4 at one level: repeat vi_ann + vi_reconstruct.
 * n_outer >= 0 runs exactly that many iterations; n_outer < 0 applies the
 * stopping rule of Sec. 3.7 (stop when e <= cfg.stop or after cfg.max_outer
 * iterations; synchronises once per iteration). n_done_host and e_last_host
 * are nullable. The call index of the k-th iteration is first_call + k, and
 * with the rule the cap counts from call 0 (first_call + k < cfg.max_outer),
 * so a loop resumed at call first_call stops where the whole loop would. */
vi_status vi_iterate(vi_ctx *ctx, int level, int n_outer, int first_call, int *n_done_host,
                     float *e_last_host);

/* Level transition (Sec. 3.6; Algorithm 4): the shift map of `level` is
 * upsampled to level-1 by nearest neighbour with its spatial components
 * doubled; shifts that leave D~ are redrawn uniformly (Philox purpose 3);
 * the occluded voxels of level-1 first take their coarse parent's values, then
 * distances are computed and level-1 is reconstructed with Eq. 4/5/9. */
vi_status vi_next_level(vi_ctx *ctx, int level);

/* Final reconstruction at level 0 (Eq. 6): each occluded voxel takes the
 * value of its best contributor u(p + phi(q*)), q* = argmin over the patches
 * containing p of the current d2 (ties: first in dt, dy, dx order). */
vi_status vi_final(vi_ctx *ctx);

/* The whole method after vi_upload: vi_prepare, then for every level from
 * the coarsest: vi_iterate with the stopping rule and vi_next_level, and
 * vi_final at level 0. */
vi_status vi_run(vi_ctx *ctx);

/* Energy of Eq. 1 at the level for the current channels and shift map:
 * E_H = sum over H of d^2 and E_H~ = the same sum over H~ (FP32 distances,
 * FP64 sums). Synchronises. Either output may be NULL. */
vi_status vi_energy(vi_ctx *ctx, int level, double *E_H_host, double *E_Ht_host);

/* The energy of vi_energy (E_H and E_H~ of Eq. 1, FP32 distances, FP64 sums)
 * for buffers the caller owns, computed without allocating any device or
 * host memory. The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc -- a process whose device memory is all
 * handed out by its own allocator under a fixed budget, or a latency-bound
 * loop that cannot take the device-wide synchronisation cudaMalloc/cudaFree
 * may cause.
 *   chans_dev: device float32 [T][H][W][C], C = 3 or 5 (the layout of
 *              vi_get_channels); phi_dev: device int32 [T][H][W][3];
 *   code_dev:  device uint8 [T][H][W] with bit 0 = occluded, bit 1 = target
 *              (the layout of vi_get_masks); voxels without bit 1 are ignored;
 *   out_dev:   device double[2] receiving (E_H, E_H~);
 *   cuda_stream: cudaStream_t the two kernels are launched on (NULL: default).
 * At most 16,777,216 voxels (W*H*T) per call: larger inputs return
 * VI_ERR_TOO_LARGE before anything runs. The scratch is one fixed 1 MiB array
 * in the library's static device memory, held by every GPU that loads the
 * library until the process exits. The first call on each device looks that
 * array's device address up (cudaGetSymbolAddress) with the device current;
 * make that first call before any stream capture. The address is kept per
 * device with the id of the CUDA context it was found in, and looked up again
 * when the device's context has changed (after a cudaDeviceReset, which
 * reloads the array: make the first call after a reset before any capture
 * too). A target counts when its source patch lies inside the video, whether
 * or not the source is in D~, exactly as in vi_energy: Eq. 1 is the energy of
 * any shift map; a source patch leaving the video gives +inf. Every call
 * shares the array, so calls that overlap on the GPU race; calls ordered on
 * one stream do not (each reads back only what it has just written).
 * Asynchronous: the result is in out_dev once the stream reaches it. Errors: VI_ERR_ARG (null
 * pointer, C, sizes), VI_ERR_TOO_LARGE, VI_ERR_CUDA. */
vi_status vi_energy_noalloc(const float *chans_dev, int C, const int32_t *phi_dev,
                            const uint8_t *code_dev, int W, int H, int T, double *out_dev,
                            void *cuda_stream);

/* Sizes of a level: dims, channels, |H|, |H~| and |D~|. Outputs nullable. */
vi_status vi_level_info(vi_ctx *ctx, int level, int *W, int *H, int *T, int *C,
                        long long *n_hole, long long *n_target, long long *n_source);

/* Channels of a level, float32 [T][H][W][C] (C from vi_level_info). */
vi_status vi_get_channels(vi_ctx *ctx, int level, float *out, int ptr_is_device);
vi_status vi_set_channels(vi_ctx *ctx, int level, const float *in, int ptr_is_device);

/* Shift map (int32 [T][H][W][3]) and distances (float32 [T][H][W]) of a level;
 * entries outside H~ read as 0 / +inf and are ignored on set. Host memory.
 * Either pointer may be NULL. */
vi_status vi_get_nnf(vi_ctx *ctx, int level, int32_t *phi_host, float *d2_host);
vi_status vi_set_nnf(vi_ctx *ctx, int level, const int32_t *phi_host, const float *d2_host);

/* Per-voxel set codes of a level, uint8 [T][H][W]: bit 0 occluded (H),
 * bit 1 target (H~), bit 2 source (D~). Host memory. */
vi_status vi_get_masks(vi_ctx *ctx, int level, uint8_t *code_host);

/* Squared patch distances (Eq. 2 / 7b) at a level for n (target, source)
 * pairs given as int32 [n][6] = (px, py, pt, sx, sy, st) in host memory;
 * +inf where the source patch leaves the video. out_host: float32 [n]. */
vi_status vi_patch_dist(vi_ctx *ctx, int level, const int32_t *pairs_host, int n, float *out_host);

/* The partial distance of Eq. 11 (Sec. 3.5) for the same pairs: target voxels
 * r with excl_host[r] != 0 (host uint8 [T][H][W] of the level, e.g. H' of the
 * onion peel) and target voxels outside the video are left out, and the sum
 * is divided by the number kept; +inf when none is kept or the source patch
 * leaves the video. Computed by the function the onion peel's search uses.
 * excl_host NULL gives vi_patch_dist. */
vi_status vi_patch_dist_partial(vi_ctx *ctx, int level, const int32_t *pairs_host, int n,
                                const uint8_t *excl_host, float *out_host);

/* The inpainted video (level-0 colour), float32 [T][H][W][3]. Known voxels
 * are the input values. Synchronises when out is host memory. */
vi_status vi_fetch_result(vi_ctx *ctx, float *rgb_out, int ptr_is_device);

/* Device-time profiling of the PatchMatch step kernel: with enable = 1 each
 * run of back-to-back step launches (the sweeps of one search, nothing else
 * between them on the context's stream) is bracketed by one pair of CUDA
 * events; step_ms sums those spans and step_timed counts the launches inside
 * them. One pair per search instead of one per launch keeps the events from
 * slowing the profiled run. */
vi_status vi_profile(vi_ctx *ctx, int enable);

/* The iterations run since the last upload that computed e (vi_iterate with
 * the stopping rule or with e_last_host): for record i < cap its level, call
 * index, e (Sec. 3.7) and the context's evaluation count after it, into the
 * nullable arrays. Returns the number of records (-1 for a null context). */
int vi_iteration_log(vi_ctx *ctx, int cap, int *level, int *call, float *e, unsigned long long *evals);

/* The context's counters (synchronises to read event times). */
vi_status vi_get_stats(vi_ctx *ctx, vi_stats *out);

/* ---------------------------------------------------------------------------
 * Checkpoint and resume (no counterpart in the paper). Between two
 * iterations of Algorithm 4's inner loop a level carries forward its channels
 * (u and the texture features of Eq. 7-9), its shift map and its distances;
 * every random draw depends only on (level, call, voxel). So a context that
 * uploaded the same clip with the same configuration and built its pyramid
 * can load a level's saved state and go on: the result is bit-identical to
 * the uninterrupted run, as long as that run went on past the saved
 * iteration. Host buffers, owned by the caller. Layout: 16 int32 of header
 * (magic "VICK", version 1, level, W, H, T, channels, zeros), then the
 * level's V x 4 channels c0..c3 (float), V x c4 (float, with texture), V x 3
 * shift components (int32 dx, dy, dt) and V distances (float), raster order.
 * ------------------------------------------------------------------------- */

/* Bytes of a saved state of `level` (0 for a bad level or no pyramid). */
size_t vi_state_bytes(vi_ctx *ctx, int level);

/* Saves the state of `level` into buf (cap >= vi_state_bytes). Synchronises.
 * Errors: VI_ERR_ARG. */
vi_status vi_save_state(vi_ctx *ctx, int level, void *buf, size_t cap);

/* Loads a saved state of `level` (same level, sizes and channels; size must
 * be exactly vi_state_bytes). With FP16 storage the copies are rebuilt.
 * Synchronises. Errors: VI_ERR_ARG (other level, clip or configuration; a
 * shift beyond 16 bits). */
vi_status vi_load_state(vi_ctx *ctx, int level, const void *buf, size_t size);

/* The rest of Algorithm 4 from call first_call of `level` (the iterations
 * there with the stopping rule, the finer levels, Eq. 6): with the state of
 * `level` saved after first_call iterations, vi_load_state + vi_resume gives
 * vi_run's result. */
vi_status vi_resume(vi_ctx *ctx, int level, int first_call);

/* ---------------------------------------------------------------------------
 * Serving (no counterpart in the paper, which runs one clip at a time). A
 * server admits submitted requests in arrival order while their device
 * footprint (vi_footprint_bytes) fits hbm_budget and one of max_slots worker
 * threads is free; each admitted request runs alone (vi_run, one context) on a
 * stream its context creates with a priority by size (requests under 2M / 8M
 * / 32M voxels first), so the GPU interleaves requests and a small one is not
 * held to the pace of a large one. The result is bit-identical to the same
 * clip run alone. Thread-safe. The caller keeps rgb, mask and rgb_out (host
 * or device memory, as ptr_is_device says) alive and untouched until the
 * request is done or failed; device inputs must be complete when submitted
 * (the worker reads them on its own stream), and a device result is complete
 * when vi_server_poll reports the request done.
 * ------------------------------------------------------------------------- */
typedef struct vi_server vi_server;

/* Errors: VI_ERR_ARG (zero budget, max_slots outside 1..256), VI_ERR_NO_DEVICE,
 * VI_ERR_OOM. The server runs on the calling thread's current device. */
vi_status vi_server_create(size_t hbm_budget, int max_slots, vi_server **out);

/* Queues one request (cfg NULL: vi_config_default); *ticket identifies it.
 * Non-blocking. Errors: VI_ERR_ARG, VI_ERR_TOO_LARGE (footprint above the
 * budget), VI_ERR_STATE (server shutting down). */
vi_status vi_server_submit(vi_server *s, const vi_config *cfg, const float *rgb, const uint8_t *mask, int W,
                           int H, int T, int ptr_is_device, float *rgb_out, uint64_t *ticket);

/* *done: 1 finished (rgb_out written), -1 failed, 0 queued or running. */
vi_status vi_server_poll(vi_server *s, uint64_t ticket, int *done);

/* Blocks until the request finishes or timeout_s elapses (timeout_s < 0:
 * no limit); *done as in vi_server_poll. */
vi_status vi_server_wait(vi_server *s, uint64_t ticket, double timeout_s, int *done);

/* Forgets a finished or failed request and returns its status (the text of
 * its error into err_buf, err_cap bytes, nullable). VI_ERR_STATE while it is
 * still queued or running. */
vi_status vi_server_release(vi_server *s, uint64_t ticket, char *err_buf, int err_cap);

/* Requests waiting, requests running, footprint bytes admitted. Nullable. */
vi_status vi_server_info(vi_server *s, int *queued, int *running, size_t *bytes_in_use);

/* Lets running requests finish, fails the queued ones, joins the workers and
 * frees the server. No other call on s may be in progress or follow. */
void vi_server_destroy(vi_server *s);

/* ---------------------------------------------------------------------------
 * Time slabs (no counterpart in the paper, whose program is not parallel):
 * the whole inpainting of one clip, as vi_run, with the targets and occluded
 * voxels of every level but the coarsest split by frames into n_slabs
 * contiguous ranges (slab r: frames [r T / n, (r + 1) T / n)), each searched
 * and reconstructed by a context of its own that holds the whole clip. The
 * coarsest level (onion peel and its iterations) runs alike in every
 * context. What a slab reads across its boundary is copied between the
 * contexts: after every Jacobi sweep the shifts and change flags of the frame
 * on each side; after a search the shifts and distances of the two frames on
 * each side; after every vote or provisional fill the channels of every
 * slab's occluded voxels to every context; and the per-voxel changes into
 * context 0, which sums e over the whole list
 * in vi_run's order. The output, the iteration counts and the evaluation
 * count are identical to vi_run's. With devices NULL all contexts run on the
 * current device on one stream (cuda_stream, or one context 0 creates),
 * which orders the copies. With devices (n_slabs entries; cuda_stream must
 * be NULL) slab r's context runs on device devices[r] on a stream of its
 * own, the copies are peer copies, and events order them: every exchange
 * waits for all work issued on every stream before it, and the next step
 * for the exchange (with device buffers devices[0] must be the current
 * device, where rgb_out lives). The result is the same either way. rgb,
 * mask, rgb_out as in vi_upload /
 * vi_fetch_result (ptr_is_device); stats_out (nullable) receives context 0's
 * counters with every slab's evaluations; exchanged_bytes (nullable) the
 * bytes copied between contexts. Errors: VI_ERR_ARG (n_slabs outside
 * 1 .. min(16, T), FP16 storage, temporal subsampling, a stream with devices,
 * a bad device; text in vi_slabs_last_error), others as vi_run.
 * ------------------------------------------------------------------------- */
vi_status vi_run_slabs(const vi_config *cfg, const float *rgb, const uint8_t *mask, int W, int H, int T,
                       int ptr_is_device, int n_slabs, float *rgb_out, vi_stats *stats_out,
                       unsigned long long *exchanged_bytes, void *cuda_stream, const int *devices);
const char *vi_slabs_last_error(void);

/* ---------------------------------------------------------------------------
 * Affine realignment: Sec. 3.4, Algorithm 2 (AlignVideo) and the UnwarpVideo
 * step that ends Algorithm 4. The paper estimates the dominant affine motion
 * between successive frames with the robust method of Odobez and Bouthemy;
 * this library's reading: a point p = (x, y) of frame n lies at A(p) = p +
 * w(p) in frame n+1, w(p) = (a0 + a1 x + a2 y, a3 + a4 x + a5 y) (theta =
 * a0..a5, pixel centres at integer coordinates), fitted by Gauss-Newton with
 * iteratively reweighted least squares (Tukey biweight, c = 4.6851 sigma) on
 * the grey level (R+G+B)/3 of the known pixels, coarse to fine over a 2x2
 * mean pyramid. All functions run on cuda_stream (NULL: the legacy default
 * stream) and synchronise it before returning. rgb: [T][H][W][3] float32;
 * mask: [T][H][W] uint8 (1 = occluded); ptr_is_device says where rgb, mask
 * and the other video buffers live (theta arrays are always host memory).
 * Errors: VI_ERR_ARG (null pointer, sizes), VI_ERR_OOM, VI_ERR_CUDA; the text
 * of the last error of the calling thread is vi_realign_last_error().
 * ------------------------------------------------------------------------- */
const char *vi_realign_last_error(void);

/* Pyramid levels the estimation uses by default: the most (up to 6) that keep
 * the smallest side of the coarsest level at least 16 pixels. */
int vi_affine_levels(int W, int H);

/* theta_{n,n+1} for n = 0 .. T-2 into theta_out[T-1][6] (host). levels = 0:
 * vi_affine_levels; iters: Gauss-Newton iterations per level (10). Occluded
 * pixels and samples touching occluded pixels take no part. */
vi_status vi_affine_estimate(const float *rgb, const uint8_t *mask, int W, int H, int T, int ptr_is_device,
                             int levels, int iters, double *theta_out, void *cuda_stream);

/* theta_{n,N_m} for every frame (host arrays): the successive motions
 * composed towards the reference frame N_m = floor(T/2) counted from 1
 * (index max(0, T/2 - 1)); inverses after it. to_ref_out[T][6]. */
vi_status vi_affine_to_reference(const double *theta_pairs, int T, double *to_ref_out);

/* AlignVideo: aligned frame n samples frame n bilinearly at
 * theta_{n,N_m}^-1(q) for every pixel q; a sample outside frame n, or whose
 * bilinear neighbours with non-zero weight include an occluded pixel, is
 * occluded in mask_out (its rgb_out value is meaningless). */
vi_status vi_affine_align(const float *rgb, const uint8_t *mask, int W, int H, int T, const double *to_ref,
                          float *rgb_out, uint8_t *mask_out, int ptr_is_device, void *cuda_stream);

/* UnwarpVideo: rgb_out = rgb where mask = 0; where mask = 1, the inpainted
 * aligned video sampled bilinearly at theta_{n,N_m}(y), clamped to the frame. */
vi_status vi_affine_unwarp(const float *rgb, const uint8_t *mask, const float *aligned_result, int W, int H,
                           int T, const double *to_ref, float *rgb_out, int ptr_is_device, void *cuda_stream);

/* Lanes-per-target autotuning (no counterpart in the paper; speed only, never
 * a result). With lanes_per_target = 0 the first rescore launch, or the
 * first PatchMatch step launch with the change-flag rule on (k >= 3; earlier
 * sweeps skip no candidate and would favour other choices), of a kernel
 * family for a target count (per device, channels,
 * storage, quarter-octave bucket of the count) is run once with every lane
 * group size in {1, 2, 4, 8} (and the warp-shared form, 32, for the
 * step kernels), timed, and the fastest is kept for the
 * process. vi_tune_export writes the table as text lines
 * "device family c5 fp16 bucket lanes" (family 0 step, 1 batch step, 2
 * rescore, 3 batch rescore) into buf (cap bytes, NUL-terminated, truncated
 * if short; buf may be NULL) and returns the bytes needed including the NUL.
 * vi_tune_import adds such lines to the table (a profiler, which serialises
 * the timing launches, can then run the choices of an unprofiled run).
 * Errors: VI_ERR_ARG on a malformed line (nothing imported). */
int vi_tune_export(char *buf, int cap);
vi_status vi_tune_import(const char *text);

/* ---------------------------------------------------------------------------
 * Batches: many clips, one launch per step.
 *
 * A batch runs the same method (Algorithm 4 without realignment) on many
 * clips of different sizes at once. Each clip keeps its own pyramid, levels,
 * seed and stopping rule; a round (vi_batch_step) runs one search and
 * reconstruction iteration (vi_ann + vi_reconstruct) for every clip still
 * iterating, whatever its level, in single launches that cover the targets
 * and occluded voxels of all of them, then applies each clip's stopping rule,
 * level transition and final step. Clips can be added and removed between
 * rounds (continuous batching). Each clip's result is bit-identical to
 * vi_run on that clip alone with the same vi_config. All work is ordered on
 * the batch's stream; a batch is used by one thread at a time.
 * ------------------------------------------------------------------------- */
typedef struct vi_batch vi_batch;

/* Creates an empty batch. cfg: defaults for its clips (use_texture and n_pm
 * are fixed for the whole batch); cuda_stream: NULL for an own stream. */
vi_status vi_batch_create(const vi_config *cfg, void *cuda_stream, vi_batch **out);
void vi_batch_destroy(vi_batch *b);
const char *vi_batch_last_error(const vi_batch *b);

/* Adds a clip (copied, as vi_upload) and prepares it (vi_prepare: pyramid,
 * initialisation, onion peel) on the batch's stream; job_cfg (nullable: the
 * batch's cfg) sets its seed, clip tag, levels and stopping parameters.
 * *id_out receives the clip's id. */
vi_status vi_batch_add(vi_batch *b, const vi_config *job_cfg, const float *rgb, const uint8_t *mask,
                       int W, int H, int T, int ptr_is_device, int *id_out);

/* Adds n clips at once: as n calls of vi_batch_add, except that the clips'
 * uploads and preparations (pyramid, initialisation, onion peel: chains of
 * small launches and synchronisations) run concurrently, each on a stream of
 * its own from one of n_threads host threads (0: 8), and join the batch's
 * stream when all are done. The copies start after everything queued on the
 * batch's stream before the call; the call returns when every clip is
 * prepared, so the inputs may then be reused. Per clip i: job_cfgs[i]
 * (job_cfgs or job_cfgs[i] NULL: the batch's cfg), rgbs[i] / masks[i] of
 * Ws[i] x Hs[i] x Ts[i] (all host or all device memory, ptr_is_device),
 * ids_out[i] its id (-1 if it failed), status_out[i] (nullable array) its
 * status. Results are those of adding the clips one by one. Returns VI_OK, or
 * the first failing clip's status (its message in vi_batch_last_error); the
 * other clips are added regardless. The paper has no counterpart (batching
 * serves many clips on one GPU). */
vi_status vi_batch_add_many(vi_batch *b, int n, const vi_config *const *job_cfgs, const float *const *rgbs,
                            const uint8_t *const *masks, const int *Ws, const int *Hs, const int *Ts,
                            int ptr_is_device, int n_threads, int *ids_out, vi_status *status_out);

/* One round for every iterating clip (synchronises once). *n_active (nullable)
 * receives the number of clips still iterating afterwards. */
vi_status vi_batch_step(vi_batch *b, int *n_active);

/* Rounds until no clip is iterating. */
vi_status vi_batch_run(vi_batch *b);

/* *done: 1 finished, 0 iterating, -1 failed; *level: its current level. */
vi_status vi_batch_poll(vi_batch *b, int id, int *done, int *level);

/* The inpainted video of a finished clip (as vi_fetch_result). */
vi_status vi_batch_fetch(vi_batch *b, int id, float *rgb_out, int ptr_is_device);

/* Releases a clip's device state. */
vi_status vi_batch_remove(vi_batch *b, int id);

/* A clip's counters (as vi_get_stats). */
vi_status vi_batch_clip_stats(vi_batch *b, int id, vi_stats *out);

/* The context behind a clip of the batch, for inspecting and injecting its
 * state between rounds with the single-clip calls (vi_level_info,
 * vi_get/set_channels, vi_get/set_nnf, vi_get_masks at the level vi_batch_poll
 * reports), e.g. to compare one batch round with the oracle's search and vote
 * on the same state. *call_out (nullable) receives the clip's iteration index
 * at its level: its next round is Algorithm 4's iteration `call` there (the
 * Philox tag of its random search). The batch keeps ownership: the handle is
 * valid until the clip is removed, and must not be destroyed, uploaded to or
 * run through vi_run. Errors: VI_ERR_ARG (unknown clip). */
vi_status vi_batch_clip_ctx(vi_batch *b, int id, vi_ctx **ctx_out, int *call_out);

/* Batch counters: patch-distance evaluations (batch launches plus the own
 * launches of every clip added so far, removed ones included), source voxels
 * gathered by the batch step launches, rounds.
 * Synchronises. Outputs nullable. */
vi_status vi_batch_get_stats(vi_batch *b, unsigned long long *evals, unsigned long long *gathered,
                             unsigned long long *rounds);

/* FP16 screening counters of the batch step launches (storage 1): FP16
 * source voxels gathered, candidates screened, candidates passed on to the
 * FP32 distance. All zero with storage 0. Synchronises. Outputs nullable. */
vi_status vi_batch_screen_stats(vi_batch *b, unsigned long long *gathered_h, unsigned long long *screened,
                                unsigned long long *passed);

/* Device-time profiling of the batch PatchMatch step launches (events on the
 * batch's stream around each launch), and its totals since creation: summed
 * milliseconds and the evaluations those launches made. Synchronises. */
vi_status vi_batch_profile(vi_batch *b, int enable);
vi_status vi_batch_step_time(vi_batch *b, double *step_ms, unsigned long long *step_evals);

#ifdef __cplusplus
}
#endif

#endif /* VI_H */
