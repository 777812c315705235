// Tiled substep kernels (TMA-staged shared-memory plane ring, register
// sliding along z).  Internal to libgbfd.
#pragma once

#include <cuda.h>

#include "kernels.cuh"

namespace gbfd {

// One entry of a tile table searched by the autotuner.
struct TileConfig {
    int tx, ty;  // xy tile (threads per CTA = tx * ty, one point each per plane)
    int zc;      // planes streamed per CTA
    int ns;      // plane slots in the shared-memory ring
    int px;      // points per thread along x (1, or 2 with paired loads)
    int pk;      // 0: scalar arithmetic; n > 0: packed FP32x2 arithmetic with
                 // n output planes per loop iteration
    int tm;      // 1: in-plane work at plane arrival, results carried through TMEM
    int lag;     // 1: output planes finished three planes behind the in-plane work
};

// Number of z-chunk lengths offered per (tx, ty, ns) variant; table index
// i is variant i / kZcChoices with the (i % kZcChoices)-th chunk length.
constexpr int kZcChoices = 5;

// FP32 tile table (55-point form; the 19-point form runs the two-plane
// packed kernel for variants 1-4):
//   0  one point per thread, 32 x 8
//   1  two points per thread, packed FP32x2 arithmetic, two output planes
//      per loop iteration, in-plane arms of the arriving plane
//   2  output planes finished three planes behind the in-plane work, each
//      plane's x/y arm differences feeding the z-paired mixed terms of the
//      planes around it, pending right-hand sides in registers, two steps
//      per iteration
//   3  the same with one step per iteration
//   4  the same as 2 with the pending right-hand sides in TMEM (default;
//      on whole tiles with equal spacing and five unforced fields it runs an
//      instantiation per RK3 substep, the substep and the grid-extent test
//      fixed at compile time)
//   5  the same as 4 compiled for three CTAs per SM (168 registers; slower:
//      13.3 against 19.2 G updates/s at 256^3, spills and still two CTAs per
//      SM, whose shared memory the ring fills; kept as the check that its
//      TMEM accesses are right since the warps are reconverged before them)
//   6  the same as 4 with the x-neighbour pairs of the x arms taken from the
//      neighbouring lanes by warp shuffles instead of paired shared loads
//      (tiled_shfl.cu)
constexpr int kVarPx1 = 0, kVarPacked = 1, kVarLagReg = 2, kVarLagReg1 = 3, kVarLagTm = 4,
              kVarLagTmCap = 5, kVarLagTmShfl = 6;
constexpr int kDefaultF32 = kVarLagTm * kZcChoices;

// Default FP64 table entry (see tiled_f64.cu): the one-point kernel with the
// output lagged three planes behind the in-plane work (z-paired Eq. 8 terms
// from each centre plane's own differences), 16 x 8 tiles, a 5-slot ring for
// three CTAs per SM, z-chunks of 40: 0.622 against 0.554 G updates/s for the
// one-point kernel that reads every stencil point (entry 5) at 256^3; the
// FP64 pipe is the bound.
constexpr int kDefaultF64 = 5 * kZcChoices;

// Tile tables per storage width (4 = FP32 storage, 8 = FP64 storage).
int tiled_config_count(int sbytes);
TileConfig tiled_config(int sbytes, int i);

// Encoded TMA descriptors of the state buffers, cached per context.
struct TmapCache {
    static constexpr int kEntries = 16;
    struct Entry {
        const void *base;
        int cfg;
        int nf;
        bool valid;
        CUtensorMap map;
    } e[kEntries];
    int next;
};

// Table variant 6 (FP32 storage and arithmetic, 55-point form).
cudaError_t launch_lag_shfl(const StateBufs &b, const Coef<float> &c, const RKStage &st, int nf,
                            int zc, int cfg_key, int *dev_error, TmapCache *cache,
                            cudaStream_t stream, int *launches);

template <class TS, class TW, class TA>
cudaError_t launch_substep_tiled(const StateBufs &b, const Coef<TS> &c, const RKStage &st, int nf,
                                 int form, int cfg, int *dev_error, TmapCache *cache,
                                 cudaStream_t stream, int *launches);

}  // namespace gbfd
