// Second pass of the 19-point form (Algorithm 3, Eqs. 14-16 / Appendix A),
// tiled, FP32 storage and arithmetic:
//   w_i   <- w_i + dt (nu/3) d_i(div u),
//   out_i <- out_i + beta dt (nu/3) d_i(div u),      i = x, y, z,
// with d_i the first derivative of Eq. 6 applied to the divergence that the
// first pass stored (Eq. 9; the i = j term is D1 o D1, the paper's "slight
// error").
//
// A CTA owns a TX x TY column and streams it along z over zc output planes.
// Each z-plane of the divergence, tile plus 3-cell halo, arrives by one TMA
// copy into a ring of NS small shared-memory slots; the x and y arms come
// from there as aligned pairs (two points per thread, packed FP32x2
// arithmetic), the z arms from the thread's own column held in registers.
// The six updated values are read and written with coalesced pair accesses
// (the outputs also refresh their periodic x/y ghost copies).  Only the
// divergence needs a halo, so each point's divergence is read from HBM once.
#pragma once

#include "tiled2_impl.cuh"

namespace gbfd {
namespace pass2 {

template <int TX, int TY, int NS>
struct Ring {
    static constexpr int BX = TX + 2 * GX;
    static constexpr int BY = TY + 2 * GY;
    static constexpr int SLOT_BYTES = BX * BY * 4;
    static constexpr int SLOT_PITCH = (SLOT_BYTES + 127) / 128 * 128;
    static constexpr int SLOT_ELEMS = SLOT_PITCH / 4;
    static constexpr int BAR_OFF = NS * SLOT_PITCH;
    static constexpr int BYTES = BAR_OFF + NS * 8;
};

template <int TX, int TY, int NS>
__global__ void __launch_bounds__((TX / 2) * TY) k_pass2_tiled(
    const __grid_constant__ CUtensorMap dmap, float *__restrict__ out, float *__restrict__ w,
    const Layout Ls, const Layout Lw, const Coef<float> c, const RKStage st, const int zc,
    const int tiles_x, int *__restrict__ dev_error)
{
    using RG = Ring<TX, TY, NS>;
    using P = tiled2::PairOps<float>;
    using V = float2;
    using tiled::mbar_wait;
    constexpr int BX = RG::BX, NTX = TX / 2;
    static_assert(NS >= 8, "the ring holds the seven planes of the z stencil plus one ahead");
    extern __shared__ __align__(128) unsigned char smem[];
    const float *sm = reinterpret_cast<const float *>(smem);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + RG::BAR_OFF);
    tiled2::init_barriers(bars, NS);

    const int x0 = (blockIdx.x % tiles_x) * TX;
    const int y0 = (blockIdx.x / tiles_x) * TY;
    const int z0 = blockIdx.y * zc;
    const int nout = min(zc, Ls.nz - z0);
    const int nplanes = nout + 2 * R;
    const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
    const int x = x0 + 2 * tx, y = y0 + ty;
    const bool valid0 = (x < Ls.nx) && (y < Ls.ny);  // nx % 4 == 0: x + 1 valid with x
    const int toff = (ty + GY) * BX + (2 * tx + GX);

    // local plane j is grid plane z0 - 3 + j, slot j % NS, phase (j / NS) & 1
    int issued = 0;
    auto issue = [&](int j) {
        const int z = zplane(Ls, z0 - R + j) + Ls.gz;  // TMA z coordinate
        const int slot = j % NS;
        tiled::mbar_expect_tx(&bars[slot], RG::SLOT_BYTES);
        tiled::tma_load_4d(smem + slot * RG::SLOT_PITCH, &dmap, &bars[slot], x0, y0, z, 0);
    };
    if (threadIdx.x == 0) {
        tiled::fence_proxy_async();
#pragma unroll 1
        for (int j = 0; j < NS && j < nplanes; ++j)
            issue(j);
        issued = min(NS, nplanes);
    }

    bool timeout = false;
    int waited = 0;
    // the column's divergence at local planes o .. o + 6 (output plane o's
    // z stencil), both points
    V col[7];
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) {
        if (!mbar_wait(&bars[j % NS], (j / NS) & 1))
            timeout = true;
        col[j] = *reinterpret_cast<const V *>(sm + (j % NS) * RG::SLOT_ELEMS + toff);
    }
    waited = 2 * R;

    const V NEG1 = P::bc(-1.f);
    const float sdt = (float)(st.dt * st.nu3);            // dt nu / 3
    const float sbd = (float)(st.beta * st.dt * st.nu3);  // beta dt nu / 3
    long long go_s = (long long)z0 * Ls.plane + (long long)(y + GY) * Ls.P + (x + GX);
    long long go_w = (long long)z0 * Lw.plane + (long long)(y + GY) * Lw.P + (x + GX);
    long long gdx = 0, gdy = 0;
    if (x < GX)
        gdx = Ls.nx;
    else if (x >= Ls.nx - GX)
        gdx = -Ls.nx;
    if (y < GY)
        gdy = (long long)Ls.ny * Ls.P;
    else if (y >= Ls.ny - GY)
        gdy = -(long long)Ls.ny * Ls.P;

#pragma unroll 1
    for (int o = 0; o < nout; ++o) {
        // every thread is done with iteration o - 1, whose centre was plane
        // o + 2: the slots of planes <= o + 2 take planes up to o + 2 + NS
        if (__syncthreads_or(timeout))
            break;
        if (threadIdx.x == 0) {
            tiled::fence_proxy_async();
            const int jend = min(o + R + NS, nplanes);
#pragma unroll 1
            for (int j = issued; j < jend; ++j)
                issue(j);
            issued = max(issued, jend);
        }
        const int jn = o + 2 * R;  // the plane entering the z window
        if (!mbar_wait(&bars[jn % NS], (jn / NS) & 1))
            timeout = true;
        waited = jn + 1;
        const int cb = ((o + R) % NS) * RG::SLOT_ELEMS + toff;  // centre plane
        col[6] = *reinterpret_cast<const V *>(sm + (jn % NS) * RG::SLOT_ELEMS + toff);
        auto ld2 = [&](int dy, int dx) -> V {
            return *reinterpret_cast<const V *>(sm + cb + dy * BX + dx);
        };
        // x arms of both points from the pairs at -4, -2, +2, +4 and the centre
        const V m4 = ld2(0, -4), m2 = ld2(0, -2), p2 = ld2(0, 2), p4 = ld2(0, 4);
        const V cc = col[3];
        const V h1 = P::mk(cc.y - m2.y, p2.x - cc.x);
        const V h2 = P::fma(m2, NEG1, p2);
        const V h3 = P::mk(p2.y - m4.y, p4.x - m2.x);
        V g[3];
        g[0] = P::fma(P::bc(c.D1(0, 3)), h3,
                      P::fma(P::bc(c.D1(0, 2)), h2, P::mul(P::bc(c.D1(0, 1)), h1)));
        V gy, gz;
#pragma unroll
        for (int k = 1; k <= 3; ++k) {
            const V dy = P::fma(ld2(-k, 0), NEG1, ld2(k, 0));
            const V dz = P::fma(col[3 - k], NEG1, col[3 + k]);
            gy = k == 1 ? P::mul(P::bc(c.D1(1, k)), dy) : P::fma(P::bc(c.D1(1, k)), dy, gy);
            gz = k == 1 ? P::mul(P::bc(c.D1(2, k)), dz) : P::fma(P::bc(c.D1(2, k)), dz, gz);
        }
        g[1] = gy;
        g[2] = gz;
        if (valid0) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if (!st.last) {
                    V *wp = reinterpret_cast<V *>(w + (1 + i) * Lw.fpitch + go_w);
                    *wp = P::fma(P::bc(sdt), g[i], *wp);
                }
                float *op = out + (1 + i) * Ls.fpitch + go_s;
                const V o2 = P::fma(P::bc(sbd), g[i], *reinterpret_cast<const V *>(op));
                *reinterpret_cast<V *>(op) = o2;
                if (gdx)
                    *reinterpret_cast<V *>(op + gdx) = o2;
                if (gdy) {
                    *reinterpret_cast<V *>(op + gdy) = o2;
                    if (gdx)
                        *reinterpret_cast<V *>(op + gdy + gdx) = o2;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 6; ++k)
            col[k] = col[k + 1];
        go_s += Ls.plane;
        go_w += Lw.plane;
    }
    const bool bad = __syncthreads_or(timeout);
    if (bad && threadIdx.x == 0) {
        atomicExch(dev_error, 1);
        // drain the copies still in flight into this CTA's shared memory
        for (int j = waited; j < issued; ++j)
            (void)mbar_wait(&bars[j % NS], (j / NS) & 1);
    }
}

}  // namespace pass2

// The tiled second pass for FP32 storage and arithmetic (32 x 8 tiles, two
// points per thread); its z-chunk is the first pass's.
inline cudaError_t launch_pass2_tiled(const StateBufs &b, const Coef<float> &c, const RKStage &st,
                                      int zc, int *dev_error, TmapCache *cache,
                                      cudaStream_t stream, int *launches)
{
    constexpr int TX = 32, TY = 8, NS = 8;
    // walls in z: the divergence's ghost planes first (its mirror is even)
    cudaError_t e = launch_fill_ghosts_z(b.div, b.Ls, 1, 0, stream, launches);
    if (e != cudaSuccess)
        return e;
    CUtensorMap *map = nullptr;
    if (!get_state_tmap(cache, b.div, b.Ls, 1, TX, TY, 2000, &map))
        return cudaErrorInvalidValue;
    const int tiles_x = (b.Ls.nx + TX - 1) / TX;
    const int tiles_y = (b.Ls.ny + TY - 1) / TY;
    const dim3 grid(tiles_x * tiles_y, (b.Ls.nz + zc - 1) / zc);
    using RG = pass2::Ring<TX, TY, NS>;
    auto kern = pass2::k_pass2_tiled<TX, TY, NS>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, RG::BYTES);
    if (e != cudaSuccess)
        return e;
    kern<<<grid, (TX / 2) * TY, RG::BYTES, stream>>>(*map, (float *)b.out, (float *)b.w, b.Ls,
                                                    b.Lw, c, st, zc, tiles_x, dev_error);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace gbfd
