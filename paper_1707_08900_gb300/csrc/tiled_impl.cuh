// Tiled fused substep (Algorithm 2; first pass of Algorithm 3 when MIXED is
// false), GB300 design:
//
// * A CTA owns a TX x TY column of the grid and streams it along z over
//   `zc` output planes.  Each plane of all NF fields, tile plus 3-cell halo
//   ((TX+8) x (TY+6) values, x halo widened to 4 for the 16-byte TMA rule),
//   arrives in shared memory by ONE 4D TMA copy (x, y, z, field) into a ring
//   of NS slots, completion signalled on a per-slot mbarrier.  The padded
//   layout keeps every box in bounds (periodic ghosts in x and y; z planes
//   are fetched by wrapped index).
// * The paper's 55-point kernel kept a (tau+2R)^3 cube per block and was
//   latency-bound by it on Kepler; here the ring holds only the 7 planes
//   the stencil spans plus prefetch, and the values on the thread's own
//   z-column (the z-axial stencil arms of every field) slide through
//   registers, so each plane is read from shared memory at the in-plane and
//   diagonal points only.
// * One thread per point of the plane; u-tilde and the outputs are read and
//   written straight from/to HBM with whole-sector (128-byte aligned) warp
//   accesses; outputs near the periodic edges also refresh the ghost copies.
// * Every mbarrier wait is bounded (about 2 s); a wait that gives up sets the
//   device error word, all threads leave together (__syncthreads_or) after
//   draining the copies still in flight.
#pragma once

#include "stencil.cuh"
#include "tiled.cuh"

namespace gbfd {

namespace tiled {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the phase with the given parity: gives up after ~2 s.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity))
            return true;
        if (global_ns() - t0 > 2000000000ull)
            return false;
    }
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int c0, int c1, int c2, int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

// Accessor over the plane ring: dz selects the plane, (dy, dx) the offset in
// it; the thread's own z-column comes from the sliding register window.
template <class TS, int NF, int BX, int FSTRIDE>
struct RingAcc {
    const TS *sb[7];  // this thread's centre in planes o..o+6 (dz = -3..3)
    TS col[NF][7];    // centre values, dz = -3..3
    __device__ __forceinline__ TS operator()(int f, int dz, int dy, int dx) const
    {
        if (dx == 0 && dy == 0)
            return col[f][dz + 3];
        return sb[dz + 3][f * FSTRIDE + dy * BX + dx];
    }
};

template <class TS, class TW, class TA, int NF, bool MIXED, int TX, int TY, int NS>
__global__ void __launch_bounds__(TX *TY) k_substep_tiled(
    const __grid_constant__ CUtensorMap tmap, TS *__restrict__ out, TW *__restrict__ w,
    TS *__restrict__ divf, const Layout Ls, const Layout Lw, const Coef<TS> c, const RKStage st,
    const int zc, const int tiles_x, int *__restrict__ dev_error)
{
    constexpr int BX = TX + 2 * GX;
    constexpr int BY = TY + 2 * GY;
    constexpr int FSTRIDE = BX * BY;
    constexpr int SLOT_BYTES = NF * FSTRIDE * (int)sizeof(TS);
    constexpr int SLOT_PITCH = (SLOT_BYTES + 127) / 128 * 128;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NS * SLOT_PITCH);

    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int x0 = (blockIdx.x % tiles_x) * TX;
    const int y0 = (blockIdx.x / tiles_x) * TY;
    const int z0 = blockIdx.y * zc;
    const int nz = Ls.nz;
    const int nout = min(zc, nz - z0);
    const int nplanes = nout + 2 * R;
    const int x = x0 + tx, y = y0 + ty;
    const bool valid = (x < Ls.nx) && (y < Ls.ny);
    const int toff = (ty + GY) * BX + (tx + GX);

    if (threadIdx.x == 0) {
#pragma unroll 1
        for (int i = 0; i < NS; ++i)
            mbar_init(&bars[i], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // local plane j is grid plane z0 - 3 + j (wrapped); it lives in slot j % NS
    // and completes phase j / NS of that slot's barrier.
    int issued = 0;
    auto issue = [&](int j) {
        int z = z0 - R + j;
        z = zplane(Ls, z) + Ls.gz;  // TMA z coordinate
        const int slot = j % NS;
        mbar_expect_tx(&bars[slot], SLOT_BYTES);
        tma_load_4d(smem + slot * SLOT_PITCH, &tmap, &bars[slot], x0, y0, z, 0);
    };
    if (threadIdx.x == 0) {
#pragma unroll 1
        for (int j = 0; j < NS - 1 && j < nplanes; ++j)
            issue(j);
        issued = min(NS - 1, nplanes);
    }

    RingAcc<TS, NF, BX, FSTRIDE> A;
    bool timeout = false;
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) {
        if (!mbar_wait(&bars[j % NS], (j / NS) & 1))
            timeout = true;
        const TS *sp = reinterpret_cast<const TS *>(smem + (j % NS) * SLOT_PITCH) + toff;
#pragma unroll
        for (int f = 0; f < NF; ++f)
            A.col[f][j] = sp[f * FSTRIDE];
    }

    const TA alpha = (TA)st.alpha, beta = (TA)st.beta, dt = (TA)st.dt;
    int waited = 2 * R;
#pragma unroll 1
    for (int o = 0; o < nout; ++o) {
        // all threads are done with plane o-1: its slot is free, and a
        // timeout seen by any thread ends the CTA for everyone
        if (__syncthreads_or(timeout))
            break;
        if (threadIdx.x == 0) {
            const int j = o + NS - 1;
            if (j < nplanes) {
                fence_proxy_async();
                issue(j);
                issued = j + 1;
            }
        }
        const int jn = o + 2 * R;
        if (!mbar_wait(&bars[jn % NS], (jn / NS) & 1))
            timeout = true;
        waited = jn + 1;
#pragma unroll
        for (int k = 0; k < 7; ++k)
            A.sb[k] = reinterpret_cast<const TS *>(smem + ((o + k) % NS) * SLOT_PITCH) + toff;
#pragma unroll
        for (int f = 0; f < NF; ++f)
            A.col[f][6] = A.sb[6][f * FSTRIDE];

        if (valid) {
            const int z = z0 + o;
            TW wv[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f)
                wv[f] = st.first ? (TW)0 : w[lidx(Lw, f, z, y, x)];
            PointDerivs<TS> d;
            gather_derivs<TS, NF, MIXED>(A, c, d);
            TS r[5];
            rhs_point<TS, NF>(d, c, r);
            if (st.fo.on) {
                const TS fc = forcing_cos<TS>(st.fo, x, y, z);
#pragma unroll
                for (int i = 0; i < 3; ++i)
                    r[1 + i] += (TS)st.fo.amp[i] * fc;
            }
            if (!MIXED) {
                const TS div = d.gu[0][0] + d.gu[1][1] + d.gu[2][2];
                store_ghosted(divf, Ls, 0, z, y, x, div);
            }
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                TS ov;
                rk3_update<TA, TW, TS>(st.first, alpha, beta, dt, (TA)r[f], A.col[f][3], wv[f], ov);
                if (!st.last)
                    w[lidx(Lw, f, z, y, x)] = wv[f];
                store_ghosted(out, Ls, f, z, y, x, ov);
            }
        }
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int k = 0; k < 6; ++k)
                A.col[f][k] = A.col[f][k + 1];
    }
    if (__syncthreads_or(timeout)) {
        if (threadIdx.x == 0) {
            atomicExch(dev_error, 1);
            // drain copies still in flight into this CTA's shared memory
            for (int j = waited; j < issued; ++j)
                (void)mbar_wait(&bars[j % NS], (j / NS) & 1);
        }
        __syncthreads();
    }
}

template <int NF, class TS, int TX, int TY, int NS>
constexpr int smem_bytes()
{
    return NS * ((NF * (TX + 2 * GX) * (TY + 2 * GY) * (int)sizeof(TS) + 127) / 128 * 128) +
           NS * 8;
}

}  // namespace tiled

// Encode (or fetch from the cache) the 4D tensor map of a padded state
// buffer for a TX x TY tile: dims (X, Y, z, field), box (TX+8, TY+6, 1, NF).
bool get_state_tmap(TmapCache *cache, const void *origin, const Layout &L, int nf, int tx, int ty,
                    int cfg_key, CUtensorMap **out);
// Tensor map of the interior tile only (no halo): box (TX, TY, 1, NF), used
// for the u-tilde buffer.
bool get_tile_tmap(TmapCache *cache, const void *origin, const Layout &L, int nf, int tx, int ty,
                   int cfg_key, CUtensorMap **out);

template <class TS, class TW, class TA, int TX, int TY, int NS>
cudaError_t launch_tiled_cfg(const StateBufs &b, const Coef<TS> &c, const RKStage &st, int nf,
                             int form, int zc, int cfg_key, int *dev_error, TmapCache *cache,
                             cudaStream_t stream, int *launches)
{
    CUtensorMap *map = nullptr;
    if (!get_state_tmap(cache, b.in, b.Ls, nf, TX, TY, cfg_key, &map))
        return cudaErrorInvalidValue;
    const int tiles_x = (b.Ls.nx + TX - 1) / TX;
    const int tiles_y = (b.Ls.ny + TY - 1) / TY;
    const dim3 grid(tiles_x * tiles_y, (b.Ls.nz + zc - 1) / zc);
    const dim3 block(TX * TY);
    TS *out = (TS *)b.out;
    TW *w = (TW *)b.w;
    TS *divf = (TS *)b.div;
    cudaError_t e;
#define GBFD_LAUNCH(NFV, MIX)                                                                     \
    do {                                                                                          \
        auto kern = tiled::k_substep_tiled<TS, TW, TA, NFV, MIX, TX, TY, NS>;                     \
        constexpr int sm = tiled::smem_bytes<NFV, TS, TX, TY, NS>();                              \
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);          \
        if (e != cudaSuccess)                                                                     \
            return e;                                                                             \
        kern<<<grid, block, sm, stream>>>(*map, out, w, divf, b.Ls, b.Lw, c, st, zc, tiles_x,     \
                                          dev_error);                                             \
    } while (0)
    if (form == 0) {
        if (nf == 5)
            GBFD_LAUNCH(5, true);
        else
            GBFD_LAUNCH(4, true);
    } else {
        if (nf == 5)
            GBFD_LAUNCH(5, false);
        else
            GBFD_LAUNCH(4, false);
    }
#undef GBFD_LAUNCH
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace gbfd
