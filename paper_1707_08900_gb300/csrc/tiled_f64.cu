// Tiled substep instantiations with FP64 storage and arithmetic.
#include "tiled_impl.cuh"

namespace gbfd {

template <class TS, class TW, class TA>
cudaError_t launch_substep_tiled(const StateBufs &b, const Coef<TS> &c, const RKStage &st, int nf,
                                 int form, int cfg, int *dev_error, TmapCache *cache,
                                 cudaStream_t stream, int *launches)
{
    const int idx = cfg < 0 ? 0 : cfg;
    const TileConfig t = tiled_config(8, idx);
    const int v = idx / kZcChoices;
    cudaError_t e;
    if (v == 0)
        e = launch_tiled_cfg<TS, TW, TA, 32, 4, 8>(b, c, st, nf, form, t.zc, v, dev_error, cache,
                                                   stream, launches);
    else
        e = launch_tiled_cfg<TS, TW, TA, 16, 8, 8>(b, c, st, nf, form, t.zc, v, dev_error, cache,
                                                   stream, launches);
    if (e != cudaSuccess || form == 0)
        return e;
    return launch_pass2_simple<TS, TW, TA>(b, c, st, stream, launches);
}

template cudaError_t launch_substep_tiled<double, double, double>(const StateBufs &,
                                                                  const Coef<double> &,
                                                                  const RKStage &, int, int, int,
                                                                  int *, TmapCache *,
                                                                  cudaStream_t, int *);

}  // namespace gbfd
