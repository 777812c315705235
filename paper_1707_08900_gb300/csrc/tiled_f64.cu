// Tiled substep instantiations with FP64 storage and arithmetic (FP64 tile
// table): 0, 1 the one-point-per-thread kernel on 32 x 4 and 16 x 8 tiles;
// 2-4 the two-point kernel on point pairs (scalar FP64 operations in pairs)
// with the z-paired Eq. 8 terms accumulated forward from each arriving plane,
// on 32 x 4 tiles with one or two output planes per iteration and on 32 x 8;
// 5 (the default) the one-point kernel with output planes finished three
// planes behind the in-plane work (tiled6_impl.cuh) on 16 x 8 tiles, a
// 5-slot ring, three CTAs per SM.  Forced steps (Sect. 6 forcing) of
// variants 1-4 run variant 0 (which has the forcing term); the 19-point form
// of variant 5 runs variant 1.
#include "tiled6_impl.cuh"

namespace gbfd {

template <class TS, class TW, class TA>
cudaError_t launch_substep_tiled(const StateBufs &b, const Coef<TS> &c, const RKStage &st, int nf,
                                 int form, int cfg, int *dev_error, TmapCache *cache,
                                 cudaStream_t stream, int *launches)
{
    const int idx = cfg < 0 ? kDefaultF64 : cfg;
    const TileConfig t = tiled_config(8, idx);
    int v = idx / kZcChoices;
    if (form != 0 && v == 5)
        v = 1;
    if (st.fo.on && v != 5)
        v = 0;
    cudaError_t e;
    switch (v) {
    case 0:
        e = launch_tiled_cfg<TS, TW, TA, 32, 4, 8>(b, c, st, nf, form, t.zc, v, dev_error, cache,
                                                   stream, launches);
        break;
    case 1:
        e = launch_tiled_cfg<TS, TW, TA, 16, 8, 8>(b, c, st, nf, form, t.zc, v, dev_error, cache,
                                                   stream, launches);
        break;
    case 2:
        e = launch_px2_cfg<TS, TW, TA, 32, 4, 6, true, 1, 1, false, false, false, 3>(
            b, c, st, nf, form, t.zc, v, dev_error, cache, stream, launches);
        break;
    case 3:
        e = launch_px2_cfg<TS, TW, TA, 32, 4, 5, true, 2, 1, false, false, false, 3>(
            b, c, st, nf, form, t.zc, v, dev_error, cache, stream, launches);
        break;
    case 4:
        e = launch_px2_cfg<TS, TW, TA, 32, 8, 5, true, 1, 1, false, false, false, 3>(
            b, c, st, nf, form, t.zc, v, dev_error, cache, stream, launches);
        break;
    default:
        e = launch_lag64_cfg<16, 8, 5, 3>(b, c, st, nf, t.zc, v, dev_error, cache, stream,
                                          launches);
        break;
    }
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
