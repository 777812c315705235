// Launch interfaces of the kernel translation units (internal to libgbfd).
#pragma once

#include "common.cuh"

namespace gbfd {

// The body force f of Eq. 2 for the current time step: the non-helical
// forcing of Sect. 6 (Eqs. 20-21), f_i(x) = amp_i cos(k.x + phi) with
// amp = N f_k.  cos(k.x + phi) = Re(tx[x] ty[y] tz[z]) from per-axis phase
// tables ta[n] = exp(2 pi i (k_a n mod N_a) / N_a), tx also carrying
// exp(i phi), so the phase is reduced exactly in integers.
struct Forcing {
    int on;
    double amp[3];
    float amp32[3];                    // amp rounded to FP32
    const double2 *tx, *ty, *tz;
    const float2 *tx32, *ty32, *tz32;  // the same tables rounded to FP32
};

template <class T>
__device__ __forceinline__ T forcing_cos(const Forcing &F, int x, int y, int z)
{
    const double2 a = __ldg(F.tx + x), b = __ldg(F.ty + y), c = __ldg(F.tz + z);
    const double re = a.x * b.x - a.y * b.y, im = a.x * b.y + a.y * b.x;
    return (T)(re * c.x - im * c.y);
}

// Per-substep scalars of Eq. 10 (and the step's forcing).
struct RKStage {
    double alpha, beta, dt;
    double nu3;  // nu / 3, used by the second pass of the 19-point form
    int first;   // substep 1: alpha_1 = 0, the old w is not read
    int last;    // substep 3: w is dead afterwards (the next step's substep 1
                 // ignores it), so it is not written
    int s;       // 0, 1, 2
    int fault_skip_plane;  // test only: CTA 0 of the tiled kernel never copies
                           // this local plane (-1: off); its bounded wait must
                           // give up and report GBFD_ERR_TIMEOUT
    Forcing fo;            // fo.on = 0: f = 0
};

inline RKStage make_stage(int s, double dt, double nu)
{
    RKStage st;
    st.alpha = RK3_ALPHA[s];
    st.beta = RK3_BETA[s];
    st.dt = dt;
    st.nu3 = nu / 3.0;
    st.first = (s == 0);
    st.last = (s == 2);
    st.fault_skip_plane = -1;
    st.s = s;
    st.fo.on = 0;
    st.fo.amp[0] = st.fo.amp[1] = st.fo.amp[2] = 0.0;
    st.fo.tx = st.fo.ty = st.fo.tz = nullptr;
    st.fo.tx32 = st.fo.ty32 = st.fo.tz32 = nullptr;
    return st;
}

template <class TS, class TW, class TA>
cudaError_t launch_substep_simple(const StateBufs &b, const Coef<TS> &c, const RKStage &st,
                                  int nf, int form, cudaStream_t stream, int *launches);

// Second pass of the 19-point form (Algorithm 3): w += dt (nu/3) grad div,
// out += beta dt (nu/3) grad div, from the stored divergence field.
template <class TS, class TW, class TA>
cudaError_t launch_pass2_simple(const StateBufs &b, const Coef<TS> &c, const RKStage &st,
                                cudaStream_t stream, int *launches);

// State copies between a compact [f][z][y][x] staging buffer (FP64 or FP32)
// and the padded layout (ghosts filled on the way in).
// Per-axis phase tables of the forcing (see Forcing): tab[0..nx) for x with
// the phase phi, then ny entries for y, then nz for z; tab32 the same in FP32.
cudaError_t launch_forcing_tables(int kx, int ky, int kz, double phi, int nx, int ny, int nz,
                                  double2 *tab, float2 *tab32, cudaStream_t stream,
                                  int *launches);

cudaError_t launch_scatter(const void *src, int src_fp64, void *dst, const Layout &L, int nf,
                           cudaStream_t stream, int *launches);
cudaError_t launch_gather(const void *src, const Layout &L, void *dst, int dst_fp64, int nf,
                          cudaStream_t stream, int *launches);

// With walls in z: fill the ghost planes of nf fields of a walled layout
// (origin = the layout's origin pointer) as parity mirrors about the wall
// points; bit f of odd_mask marks an odd field (u_z: bit 3).  No-op for
// periodic layouts.
constexpr int kWallOddMask = 1 << 3;
cudaError_t launch_fill_ghosts_z(void *origin, const Layout &L, int nf, int odd_mask,
                                 cudaStream_t stream, int *launches);

// FP64 reductions: partials per block, then one fixed-order final pass.
// out[16]: mass, ekin, umax, urms, rms[5], maxabs[5], nonfinite, (pad).
int diag_blocks(const Layout &L);
cudaError_t launch_diagnostics(const void *state, const Layout &L, int nf, double dv,
                               double *partials, int nblocks, double *out, cudaStream_t stream,
                               int *launches);

}  // namespace gbfd
