// The default FP32 kernel (lagged output, pending right-hand sides in TMEM)
// with the x-neighbour pairs of its x arms exchanged between lanes by warp
// shuffles (table variant 6), in a translation unit of its own so that it
// compiles beside the other variants.
#include "tiled4_impl.cuh"

namespace gbfd {

cudaError_t launch_lag_shfl(const StateBufs &b, const Coef<float> &c, const RKStage &st, int nf,
                            int zc, int cfg_key, int *dev_error, TmapCache *cache,
                            cudaStream_t stream, int *launches)
{
    return launch_lag_cfg<float, float, 32, 8, 8, 2, true, 1, false, true>(
        b, c, st, nf, zc, cfg_key, dev_error, cache, stream, launches);
}

}  // namespace gbfd
