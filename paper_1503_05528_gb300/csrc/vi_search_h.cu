// vi_search_h.cu -- the PatchMatch step kernels of vi_ann.cuh for FP16
// storage: every candidate is screened on the FP16 copies of the channels and
// only the ones that may beat the current best are evaluated in FP32.
#include "vi_ann.cuh"

namespace vi {

void launch_ann_step_f16(const AnnArgs &a, bool c5, cudaStream_t st) { launch_ann_step_impl<true>(a, c5, st); }

void launch_ann_step_batch_f16(const BatchClip *clips, const int *tprefix, int n, int total_targets, BatchSweep k,
                               bool c5, unsigned long long *ctr, int lanes, cudaStream_t st)
{
    launch_ann_step_batch_impl<true>(clips, tprefix, n, total_targets, k, c5, ctr, lanes, st);
}

}  // namespace vi
