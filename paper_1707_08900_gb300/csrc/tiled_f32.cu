// Tiled substep instantiations with FP32 storage and FP32 arithmetic: the
// one-point-per-thread kernel (variants 0-3), the paired-load
// two-points-per-thread kernel (variants 4-6) and the same with the two
// points' arithmetic in packed FP32x2 instructions (variants 7-10 and 13-16:
// one, two or three output planes per loop iteration, ring lengths,
// u-tilde from global memory, larger tiles) and, for the 55-point form, the
// kernel that does the in-plane work at plane arrival and carries its
// results through TMEM (variants 11-12) and the kernel that finishes output
// planes three planes behind the in-plane work (variants 17-19: two or one
// steps per iteration, pending right-hand sides in registers or, 19, the
// default, in TMEM).
#include "tiled3_impl.cuh"
#include "tiled4_impl.cuh"

namespace gbfd {

template <class TS, class TW, class TA>
cudaError_t launch_substep_tiled(const StateBufs &b, const Coef<TS> &c, const RKStage &st, int nf,
                                 int form, int cfg, int *dev_error, TmapCache *cache,
                                 cudaStream_t stream, int *launches)
{
    // default: two points per thread in packed arithmetic, 32 x 8 tile,
    // lagged output with TMEM, z-chunk 40 (the best compromise between 256^3
    // and 512^3 on GB300 in the chunk sweep: 7 chunks of a 256 column fill
    // 5.9 launch waves of 2 x 152 CTAs, 8 chunks of 32 fill 6.7)
    const int idx = cfg < 0 ? kDefaultF32 : cfg;
    const TileConfig t = tiled_config(4, idx);
    // a forced step (Sect. 6 forcing) runs on the default kernel, whatever
    // the tile table entry
    const int v = st.fo.on ? kDefaultF32 / kZcChoices : idx / kZcChoices;
    cudaError_t e;
    switch (v) {
    case 0:
        e = launch_tiled_cfg<TS, TW, TA, 32, 8, 9>(b, c, st, nf, form, t.zc, v, dev_error, cache,
                                                   stream, launches);
        break;
    case 1:
        e = launch_tiled_cfg<TS, TW, TA, 32, 4, 9>(b, c, st, nf, form, t.zc, v, dev_error, cache,
                                                   stream, launches);
        break;
    case 2:
        e = launch_tiled_cfg<TS, TW, TA, 64, 4, 9>(b, c, st, nf, form, t.zc, v, dev_error, cache,
                                                   stream, launches);
        break;
    case 3:
        e = launch_tiled_cfg<TS, TW, TA, 32, 16, 9>(b, c, st, nf, form, t.zc, v, dev_error, cache,
                                                    stream, launches);
        break;
    case 4:
        e = launch_px2_cfg<TS, TW, TA, 32, 8, 8>(b, c, st, nf, form, t.zc, v, dev_error, cache,
                                                 stream, launches);
        break;
    case 5:
        e = launch_px2_cfg<TS, TW, TA, 32, 16, 9>(b, c, st, nf, form, t.zc, v, dev_error, cache,
                                                  stream, launches);
        break;
    case 6:
        e = launch_px2_cfg<TS, TW, TA, 64, 8, 9>(b, c, st, nf, form, t.zc, v, dev_error, cache,
                                                 stream, launches);
        break;
    case 7:
        e = launch_px2_cfg<TS, TW, TA, 32, 8, 8, true>(b, c, st, nf, form, t.zc, v, dev_error,
                                                       cache, stream, launches);
        break;
    case 8:
        e = launch_px2_cfg<TS, TW, TA, 32, 8, 8, true, 2, 1, false, false, true>(
            b, c, st, nf, form, t.zc, v, dev_error, cache, stream, launches);
        break;
    case 9:
        e = launch_px2_cfg<TS, TW, TA, 32, 8, 7, true, 3>(b, c, st, nf, form, t.zc, v, dev_error,
                                                          cache, stream, launches);
        break;
    case 10:
        // five-slot ring, registers capped for three CTAs per SM
        e = launch_px2_cfg<TS, TW, TA, 32, 8, 5, true, 1, 3>(b, c, st, nf, form, t.zc, v,
                                                             dev_error, cache, stream, launches);
        break;
    case 13:
        // six-slot ring, u-tilde read from global memory, three CTAs per SM
        e = launch_px2_cfg<TS, TW, TA, 32, 8, 6, true, 1, 3, true>(b, c, st, nf, form, t.zc, v,
                                                                   dev_error, cache, stream,
                                                                   launches);
        break;
    case 14:
        // the default kernel with u-tilde read from global memory
        e = launch_px2_cfg<TS, TW, TA, 32, 8, 8, true, 2, 1, true>(b, c, st, nf, form, t.zc, v,
                                                                   dev_error, cache, stream,
                                                                   launches);
        break;
    case 15:
        e = launch_px2_cfg<TS, TW, TA, 32, 16, 8, true, 2>(b, c, st, nf, form, t.zc, v, dev_error,
                                                           cache, stream, launches);
        break;
    case 16:
        e = launch_px2_cfg<TS, TW, TA, 64, 8, 8, true, 2>(b, c, st, nf, form, t.zc, v, dev_error,
                                                          cache, stream, launches);
        break;
    case 17:
    case 18:
    case 19:
        // output planes finished three planes behind the in-plane work
        // (55-point form; the 19-point form runs the two-plane packed kernel,
        // forcing included, as variant 8 does)
        if (form != 0)
            e = launch_px2_cfg<TS, TW, TA, 32, 8, 8, true, 2, 1, false, false, true, 1>(
                b, c, st, nf, form, t.zc, v, dev_error, cache, stream, launches);
        else if (v == 17)
            e = launch_lag_cfg<TW, TA, 32, 8, 8, 2>(b, c, st, nf, t.zc, v, dev_error, cache,
                                                     stream, launches);
        else if (v == 19)
            e = launch_lag_cfg<TW, TA, 32, 8, 8, 2, true>(b, c, st, nf, t.zc, v, dev_error, cache,
                                                           stream, launches);
        else
            e = launch_lag_cfg<TW, TA, 32, 8, 8, 1>(b, c, st, nf, t.zc, v, dev_error, cache,
                                                     stream, launches);
        break;
    default:  // 11, 12
        // in-plane work at arrival, carried through TMEM (55-point form; the
        // 19-point form runs the two-plane packed kernel on the same tile)
        if (form != 0)
            e = launch_px2_cfg<TS, TW, TA, 32, 8, 8, true, 2>(b, c, st, nf, form, t.zc, v,
                                                              dev_error, cache, stream, launches);
        else if (t.ns == 4)
            e = launch_tm_cfg<32, 8, 4>(b, c, st, nf, t.zc, v, dev_error, cache, stream,
                                        launches);
        else
            e = launch_tm_cfg<32, 8, 6>(b, c, st, nf, t.zc, v, dev_error, cache, stream,
                                        launches);
        break;
    }
    if (e != cudaSuccess || form == 0)
        return e;
    return launch_pass2_simple<TS, TW, TA>(b, c, st, stream, launches);
}

template cudaError_t launch_substep_tiled<float, float, float>(const StateBufs &,
                                                               const Coef<float> &,
                                                               const RKStage &, int, int, int,
                                                               int *, TmapCache *, cudaStream_t,
                                                               int *);

}  // namespace gbfd
