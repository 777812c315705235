// Tiled substep instantiations with FP32 storage and FP32 arithmetic, one per
// variant of the FP32 tile table (tiled.cuh): the one-point-per-thread
// kernel, the two-plane packed two-point kernel, and the kernel that
// finishes output planes three planes behind the in-plane work (pending
// right-hand sides in registers, two or one steps per iteration, or in TMEM:
// the default; its warp-shuffle variant is compiled in tiled_shfl.cu).  The z-chunk length comes from the table entry; the API picks
// the default entry's chunk per grid (fp32_default_cfg in api.cu).
#include "tiled4_impl.cuh"

namespace gbfd {

template <class TS, class TW, class TA>
cudaError_t launch_substep_tiled(const StateBufs &b, const Coef<TS> &c, const RKStage &st, int nf,
                                 int form, int cfg, int *dev_error, TmapCache *cache,
                                 cudaStream_t stream, int *launches)
{
    const int idx = cfg < 0 ? kDefaultF32 : cfg;
    const TileConfig t = tiled_config(4, idx);
    // a forced step (Sect. 6 forcing) runs on the default kernel, whatever
    // the tile table entry
    const int v = st.fo.on ? kDefaultF32 / kZcChoices : idx / kZcChoices;
    cudaError_t e;
    if (v == kVarPx1) {
        e = launch_tiled_cfg<TS, TW, TA, 32, 8, 9>(b, c, st, nf, form, t.zc, v, dev_error, cache,
                                                   stream, launches);
    } else if (form != 0 || v == kVarPacked) {
        // the two-plane packed kernel: every variant of the 19-point form
        // (its first pass has no cross terms to lag), forcing included, with
        // the isotropic weights on equal spacings (19-point form)
        e = launch_px2_cfg<TS, TW, TA, 32, 8, 8, true, 2, 1, false, false, true, 1>(
            b, c, st, nf, form, t.zc, v, dev_error, cache, stream, launches);
    } else if (v == kVarLagReg) {
        e = launch_lag_cfg<TW, TA, 32, 8, 8, 2>(b, c, st, nf, t.zc, v, dev_error, cache, stream,
                                                 launches);
    } else if (v == kVarLagReg1) {
        e = launch_lag_cfg<TW, TA, 32, 8, 8, 1>(b, c, st, nf, t.zc, v, dev_error, cache, stream,
                                                 launches);
    } else if (v == kVarLagTm) {
        e = launch_lag_cfg<TW, TA, 32, 8, 8, 2, true>(b, c, st, nf, t.zc, v, dev_error, cache,
                                                    stream, launches);
    } else if (v == kVarLagTmCap) {
        e = launch_lag_cfg<TW, TA, 32, 8, 8, 2, true, 3>(b, c, st, nf, t.zc, v, dev_error, cache,
                                                       stream, launches);
    } else {
        e = launch_lag_shfl(b, c, st, nf, t.zc, v, dev_error, cache, stream, launches);
    }
    if (e != cudaSuccess || form == 0)
        return e;
    // the 19-point form's second pass: two x-adjacent points per thread
    // with pair accesses where the layout keeps pairs aligned, else one
    // point per thread.  Measured slower at 256^3 for the form: a
    // z-streaming TMA-tiled version (10.2 against 11.6 G updates/s, its
    // per-plane work too small to hide the ring's latency) and one thread
    // per z-column with the divergence sliding through registers (10.55
    // against 11.3 G with 40-plane columns, 10.54 with 16: fewer
    // independent loads in flight per thread)
    return launch_pass2_simple<TS, TW, TA>(b, c, st, stream, launches);
}

template cudaError_t launch_substep_tiled<float, float, float>(const StateBufs &,
                                                               const Coef<float> &,
                                                               const RKStage &, int, int, int,
                                                               int *, TmapCache *, cudaStream_t,
                                                               int *);

}  // namespace gbfd
