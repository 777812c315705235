// Tiled substep instantiations of the precision form: FP32 storage and
// stencils, FP64 arithmetic for the Eq. 10 register update (u-tilde stored
// in FP32, or in FP64 for the _W64 variant).  Table entries 0-3: the packed
// two-point kernel with two output planes per iteration, its FP32<->FP64
// conversions done by integer instructions (default); 4-7: the one-point
// kernel; 8-11: the packed kernel with the hardware conversions (bitwise the
// same results as 0-3); each with the four z-chunk lengths.
#include "tiled2_impl.cuh"

namespace gbfd {

template <class TS, class TW, class TA>
cudaError_t launch_substep_tiled(const StateBufs &b, const Coef<TS> &c, const RKStage &st, int nf,
                                 int form, int cfg, int *dev_error, TmapCache *cache,
                                 cudaStream_t stream, int *launches)
{
    // default: the packed kernel with integer conversions, z-chunk 32 (its
    // FP64 update binds; 40-plane chunks measured 3% slower here)
    const int idx = cfg < 0 ? 1 : cfg;
    const TileConfig t = tiled_config(4, idx % kZcChoices);
    cudaError_t e;
    // FP64 u-tilde doubles its ring: a 6-slot state ring keeps two CTAs per SM
    constexpr int NSP = sizeof(TW) == 8 ? 6 : 8;
    int v = (idx / kZcChoices) % 3;
    if (st.fo.on && v == 2)
        v = 0;  // forced steps: the packed kernel with the forcing instantiation
    if (v == 0)
        e = launch_px2_cfg<TS, TW, TA, 32, 8, NSP, true, 2, 1, false, true, true, 2>(
            b, c, st, nf, form, t.zc, 0, dev_error, cache, stream, launches);
    else if (v == 1)
        e = launch_tiled_cfg<TS, TW, TA, 32, 8, 9>(b, c, st, nf, form, t.zc, 1, dev_error, cache,
                                                   stream, launches);
    else
        e = launch_px2_cfg<TS, TW, TA, 32, 8, NSP, true, 2, 1, false, false>(
            b, c, st, nf, form, t.zc, 2, dev_error, cache, stream, launches);
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
