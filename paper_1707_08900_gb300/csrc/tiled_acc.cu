// Tiled substep instantiations of the precision form: FP32 storage and
// stencils, FP64 arithmetic for the Eq. 10 register update (u-tilde stored
// in FP32, or in FP64 for the _W64 variant).  One tile variant (32 x 8).
#include "tiled_impl.cuh"

namespace gbfd {

template <class TS, class TW, class TA>
cudaError_t launch_substep_tiled(const StateBufs &b, const Coef<TS> &c, const RKStage &st, int nf,
                                 int form, int cfg, int *dev_error, TmapCache *cache,
                                 cudaStream_t stream, int *launches)
{
    const int idx = cfg < 0 ? 0 : cfg;
    const TileConfig t = tiled_config(4, idx % kZcChoices);
    cudaError_t e = launch_tiled_cfg<TS, TW, TA, 32, 8, 9>(b, c, st, nf, form, t.zc, 0, dev_error,
                                                           cache, stream, launches);
    if (e != cudaSuccess || form == 0)
        return e;
    return launch_pass2_simple<TS, TW, TA>(b, c, st, stream, launches);
}

template cudaError_t launch_substep_tiled<float, float, double>(const StateBufs &,
                                                                const Coef<float> &,
                                                                const RKStage &, int, int, int,
                                                                int *, TmapCache *, cudaStream_t,
                                                                int *);
template cudaError_t launch_substep_tiled<float, double, double>(const StateBufs &,
                                                                 const Coef<float> &,
                                                                 const RKStage &, int, int, int,
                                                                 int *, TmapCache *, cudaStream_t,
                                                                 int *);

}  // namespace gbfd
