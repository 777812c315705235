// The default FP32 kernel (lagged output, pending right-hand sides in TMEM)
// on 32 x 16 tiles: 256 threads, one CTA per SM (table variant 7), in a
// translation unit of its own so that it compiles beside the other variants.
#include "tiled4_impl.cuh"

namespace gbfd {

cudaError_t launch_lag_tall(const StateBufs &b, const Coef<float> &c, const RKStage &st, int nf,
                            int zc, int cfg_key, int *dev_error, TmapCache *cache,
                            cudaStream_t stream, int *launches)
{
    return launch_lag_cfg<float, float, 32, 16, 8, 2, true>(b, c, st, nf, zc, cfg_key, dev_error,
                                                           cache, stream, launches);
}

}  // namespace gbfd
