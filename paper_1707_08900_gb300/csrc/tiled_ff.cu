// Tiled substep of the float-float precision form: FP32 storage and
// stencils, the Eq. 10 update in compensated FP32 pairs (common.cuh,
// rk3_update_ff), u-tilde stored in FP32.  It runs the FP32 default kernel
// (output lagged three planes, pending right-hand sides in TMEM) with the
// tile table entry's z-chunk; 55-point form only.
#include "tiled4_impl.cuh"

namespace gbfd {

template <class TS, class TW, class TA>
cudaError_t launch_substep_tiled(const StateBufs &b, const Coef<TS> &c, const RKStage &st, int nf,
                                 int form, int cfg, int *dev_error, TmapCache *cache,
                                 cudaStream_t stream, int *launches)
{
    if (form != 0)
        return cudaErrorNotSupported;
    const int idx = cfg < 0 ? kDefaultF32 : cfg;
    const TileConfig t = tiled_config(4, idx);
    return launch_lag_cfg<TW, TA, 32, 8, 8, 2, true>(b, c, st, nf, t.zc, kVarLagTm, dev_error, cache,
                                                   stream, launches);
}

template cudaError_t launch_substep_tiled<float, float, ffloat>(const StateBufs &,
                                                                const Coef<float> &,
                                                                const RKStage &, int, int, int,
                                                                int *, TmapCache *, cudaStream_t,
                                                                int *);

}  // namespace gbfd
