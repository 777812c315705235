// Simple substep kernels: one thread per grid point, every stencil value read
// from global memory (L1/L2 cached).  They are the generic path for any
// valid grid and the cross-check for the tiled kernels; the fused
// 55-point substep is Algorithm 2, the two kernels of the 19-point form are
// the two passes of Algorithm 3 (Eqs. 14-16).
#include <type_traits>

#include "kernels.cuh"
#include "stencil.cuh"

namespace gbfd {

namespace {

template <class T>
struct GlobalAcc {
    const T *__restrict__ base;  // origin of the padded state
    Layout L;
    int x, y;
    int zk[7];  // wrapped plane index for dz = -3..3
    __device__ __forceinline__ T operator()(int f, int dz, int dy, int dx) const
    {
        return __ldg(base + (long long)f * L.fpitch + (long long)zk[dz + 3] * L.plane +
                     (long long)(y + GY + dy) * L.P + (x + GX + dx));
    }
};

template <class T>
__device__ __forceinline__ GlobalAcc<T> make_acc(const T *base, const Layout &L, int x, int y,
                                                 int z)
{
    GlobalAcc<T> A;
    A.base = base;
    A.L = L;
    A.x = x;
    A.y = y;
#pragma unroll
    for (int k = -3; k <= 3; ++k) {
        A.zk[k + 3] = zplane(L, z + k);
    }
    return A;
}

// Algorithm 2 (MIXED = true) or the first pass of Algorithm 3 (MIXED = false,
// which also stores div u for the second pass).
template <class TS, class TW, class TA, int NF, bool MIXED>
__global__ void __launch_bounds__(128) k_substep_simple(const TS *__restrict__ in,
                                                        TS *__restrict__ out,
                                                        TW *__restrict__ w, TS *__restrict__ divf,
                                                        Layout Ls, Layout Lw, Coef<TS> c,
                                                        RKStage st)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= Ls.nx || y >= Ls.ny)
        return;
    GlobalAcc<TS> A = make_acc(in, Ls, x, y, z);
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
        TS div = d.gu[0][0] + d.gu[1][1] + d.gu[2][2];
        store_ghosted(divf, Ls, 0, z, y, x, div);
    }
    const TA alpha = (TA)st.alpha, beta = (TA)st.beta, dt = (TA)st.dt;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const long long iw = lidx(Lw, f, z, y, x);
        TW wv = st.first ? (TW)0 : w[iw];
        TS o;
        rk3_update<TA, TW, TS>(st.first, alpha, beta, dt, (TA)r[f], A(f, 0, 0, 0), wv, o);
        if (!st.last)
            w[iw] = wv;
        store_ghosted(out, Ls, f, z, y, x, o);
    }
}

// The divergence around one point for the second pass: the point's address
// once, its z neighbours by precomputed plane offsets (periodic wrap or
// ghost planes), the x and y neighbours by constant offsets.
template <class T>
struct DivAcc {
    const T *__restrict__ p;  // divergence at (x, y, z)
    long long P;              // row pitch
    long long dz[7];          // offset of plane z + k - 3 from plane z
    __device__ __forceinline__ T operator()(int, int kz, int ky, int kx) const
    {
        return __ldg(p + dz[kz + 3] + ky * P + kx);
    }
};

// Second pass of Algorithm 3: w += dt (nu/3) grad(div u),
// out += beta dt (nu/3) grad(div u), grad by Eq. 6 on the stored divergence.
// Every load is issued before the first store.
template <class TS, class TW, class TA>
__global__ void __launch_bounds__(128) k_pass2_simple(const TS *__restrict__ divf,
                                                      TS *__restrict__ out, TW *__restrict__ w,
                                                      Layout Ls, Layout Lw, Coef<TS> c,
                                                      RKStage st)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= Ls.nx || y >= Ls.ny)
        return;
    const long long cs = (long long)z * Ls.plane + (long long)(y + GY) * Ls.P + (x + GX);
    const long long cw = (long long)z * Lw.plane + (long long)(y + GY) * Lw.P + (x + GX);
    DivAcc<TS> A;
    A.p = divf + cs;
    A.P = Ls.P;
#pragma unroll
    for (int k = -3; k <= 3; ++k)
        A.dz[k + 3] = (long long)(zplane(Ls, z + k) - z) * Ls.plane;
    TA g[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        g[i] = (TA)d1_axis(A, 0, i, c);
    TS ov[3];
    TW wv[3];
    const bool keep_w = !st.last;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        ov[i] = out[cs + (1 + i) * Ls.fpitch];
        if (keep_w)
            wv[i] = w[cw + (1 + i) * Lw.fpitch];
    }
    const TA dt = (TA)st.dt, beta = (TA)st.beta, nu3 = (TA)st.nu3;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (keep_w)
            w[cw + (1 + i) * Lw.fpitch] = (TW)((TA)wv[i] + dt * nu3 * g[i]);
        store_ghosted(out, Ls, 1 + i, z, y, x, (TS)((TA)ov[i] + beta * dt * nu3 * g[i]));
    }
}

// Two x-adjacent points (x even, x + 1) per thread of the second pass, with
// 8- or 16-byte pair accesses.  x and x + 1 fall on the same side of every
// periodic edge (nx even), so their ghost copies are one pair too.  Each
// point's arithmetic is the one-point kernel's, in the same order.
template <class T>
struct Pair;
template <>
struct Pair<float> {
    using t = float2;
};
template <>
struct Pair<double> {
    using t = double2;
};

template <class T>
__device__ __forceinline__ typename Pair<T>::t ldg_pair(const T *p)
{
    return __ldg(reinterpret_cast<const typename Pair<T>::t *>(p));
}

// The divergence around point x + J of the pair, from preloaded pairs: the
// x row at x - 4 .. x + 5, and the y and z arms (pairs at the same x).
template <class T, int J>
struct PairDivAcc {
    using V = typename Pair<T>::t;
    const V *xrow;    // 5 pairs: x - 4, x - 2, x, x + 2, x + 4
    const V *yarm;    // 6 pairs: dy = -3..-1, 1..3
    const V *zarm;    // 6 pairs: dz = -3..-1, 1..3
    __device__ __forceinline__ T operator()(int, int kz, int ky, int kx) const
    {
        if (kz)
            return J ? zarm[kz < 0 ? kz + 3 : kz + 2].y : zarm[kz < 0 ? kz + 3 : kz + 2].x;
        if (ky)
            return J ? yarm[ky < 0 ? ky + 3 : ky + 2].y : yarm[ky < 0 ? ky + 3 : ky + 2].x;
        const int e = J + kx + 4;  // element index in the x row
        return (e & 1) ? xrow[e >> 1].y : xrow[e >> 1].x;
    }
};

template <class T>
__device__ __forceinline__ void store_pair_ghosted(T *base, const Layout &L, int f, int z, int y,
                                                   int x, typename Pair<T>::t v)
{
    using V = typename Pair<T>::t;
    const long long i0 = lidx(L, f, z, y, x);
    *reinterpret_cast<V *>(base + i0) = v;
    long long dx = 0, dy = 0;
    if (x < GX)
        dx = L.nx;
    else if (x >= L.nx - GX)
        dx = -L.nx;
    if (y < GY)
        dy = (long long)L.ny * L.P;
    else if (y >= L.ny - GY)
        dy = -(long long)L.ny * L.P;
    if (dx)
        *reinterpret_cast<V *>(base + i0 + dx) = v;
    if (dy) {
        *reinterpret_cast<V *>(base + i0 + dy) = v;
        if (dx)
            *reinterpret_cast<V *>(base + i0 + dy + dx) = v;
    }
}

template <class TS, class TW, class TA>
__global__ void __launch_bounds__(128) k_pass2_pair(const TS *__restrict__ divf,
                                                    TS *__restrict__ out, TW *__restrict__ w,
                                                    Layout Ls, Layout Lw, Coef<TS> c, RKStage st)
{
    using V = typename Pair<TS>::t;
    using VW = typename Pair<TW>::t;
    const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= Ls.nx || y >= Ls.ny)
        return;
    const long long cs = (long long)z * Ls.plane + (long long)(y + GY) * Ls.P + (x + GX);
    const long long cw = (long long)z * Lw.plane + (long long)(y + GY) * Lw.P + (x + GX);
    const TS *p = divf + cs;
    V xrow[5], yarm[6], zarm[6];
#pragma unroll
    for (int k = 0; k < 5; ++k)
        xrow[k] = ldg_pair(p + 2 * k - 4);
#pragma unroll
    for (int k = 1; k <= 3; ++k) {
        yarm[3 - k] = ldg_pair(p - k * Ls.P);
        yarm[2 + k] = ldg_pair(p + k * Ls.P);
        zarm[3 - k] = ldg_pair(p + (long long)(zplane(Ls, z - k) - z) * Ls.plane);
        zarm[2 + k] = ldg_pair(p + (long long)(zplane(Ls, z + k) - z) * Ls.plane);
    }
    const PairDivAcc<TS, 0> A0{xrow, yarm, zarm};
    const PairDivAcc<TS, 1> A1{xrow, yarm, zarm};
    TA g0[3], g1[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        g0[i] = (TA)d1_axis(A0, 0, i, c);
        g1[i] = (TA)d1_axis(A1, 0, i, c);
    }
    V ov[3];
    VW wv[3];
    const bool keep_w = !st.last;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        ov[i] = *reinterpret_cast<const V *>(out + cs + (1 + i) * Ls.fpitch);
        if (keep_w)
            wv[i] = *reinterpret_cast<const VW *>(w + cw + (1 + i) * Lw.fpitch);
    }
    const TA dt = (TA)st.dt, beta = (TA)st.beta, nu3 = (TA)st.nu3;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (keep_w) {
            VW nw;
            nw.x = (TW)((TA)wv[i].x + dt * nu3 * g0[i]);
            nw.y = (TW)((TA)wv[i].y + dt * nu3 * g1[i]);
            *reinterpret_cast<VW *>(w + cw + (1 + i) * Lw.fpitch) = nw;
        }
        V no;
        no.x = (TS)((TA)ov[i].x + beta * dt * nu3 * g0[i]);
        no.y = (TS)((TA)ov[i].y + beta * dt * nu3 * g1[i]);
        store_pair_ghosted(out, Ls, 1 + i, z, y, x, no);
    }
}

}  // namespace

template <class TS, class TW, class TA>
cudaError_t launch_substep_simple(const StateBufs &b, const Coef<TS> &c, const RKStage &st,
                                  int nf, int form, cudaStream_t stream, int *launches)
{
    const dim3 block(32, 4, 1);
    const dim3 grid((b.Ls.nx + 31) / 32, (b.Ls.ny + 3) / 4, b.Ls.nz);
    const TS *in = (const TS *)b.in;
    TS *out = (TS *)b.out;
    TW *w = (TW *)b.w;
    TS *divf = (TS *)b.div;
    if (form == 0) {
        if (nf == 5)
            k_substep_simple<TS, TW, TA, 5, true><<<grid, block, 0, stream>>>(in, out, w, divf, b.Ls,
                                                                             b.Lw, c, st);
        else
            k_substep_simple<TS, TW, TA, 4, true><<<grid, block, 0, stream>>>(in, out, w, divf, b.Ls,
                                                                             b.Lw, c, st);
        *launches += 1;
        return cudaGetLastError();
    }
    if constexpr (std::is_same<TA, ffloat>::value) {
        return cudaErrorNotSupported;  // the float-float form is 55-point only
    } else {
        if (nf == 5)
            k_substep_simple<TS, TW, TA, 5, false><<<grid, block, 0, stream>>>(in, out, w, divf,
                                                                              b.Ls, b.Lw, c, st);
        else
            k_substep_simple<TS, TW, TA, 4, false><<<grid, block, 0, stream>>>(in, out, w, divf,
                                                                              b.Ls, b.Lw, c, st);
        cudaError_t e = cudaGetLastError();
        *launches += 1;
        if (e != cudaSuccess)
            return e;
        return launch_pass2_simple<TS, TW, TA>(b, c, st, stream, launches);
    }
}

template <class TS, class TW, class TA>
cudaError_t launch_pass2_simple(const StateBufs &b, const Coef<TS> &c, const RKStage &st,
                                cudaStream_t stream, int *launches)
{
    // walls in z: the stored divergence is even about a wall; its ghost
    // planes are filled between the passes
    cudaError_t e = launch_fill_ghosts_z(b.div, b.Ls, 1, 0, stream, launches);
    if (e != cudaSuccess)
        return e;
    const dim3 block(32, 4, 1);
    // pairs of x points with 8- or 16-byte accesses when every row start
    // and field pitch keeps an even x on a pair boundary
    auto even = [](const void *q, size_t bytes) { return ((uintptr_t)q % bytes) == 0; };
    const bool pairs = b.Ls.nx % 2 == 0 && b.Ls.P % 2 == 0 && b.Ls.plane % 2 == 0 &&
                       b.Ls.fpitch % 2 == 0 && b.Lw.P % 2 == 0 && b.Lw.plane % 2 == 0 &&
                       b.Lw.fpitch % 2 == 0 && GX % 2 == 0 && even(b.div, 2 * sizeof(TS)) &&
                       even(b.out, 2 * sizeof(TS)) && even(b.w, 2 * sizeof(TW));
    if (pairs) {
        const dim3 grid((b.Ls.nx / 2 + 31) / 32, (b.Ls.ny + 3) / 4, b.Ls.nz);
        k_pass2_pair<TS, TW, TA><<<grid, block, 0, stream>>>((const TS *)b.div, (TS *)b.out,
                                                             (TW *)b.w, b.Ls, b.Lw, c, st);
    } else {
        const dim3 grid((b.Ls.nx + 31) / 32, (b.Ls.ny + 3) / 4, b.Ls.nz);
        k_pass2_simple<TS, TW, TA><<<grid, block, 0, stream>>>((const TS *)b.div, (TS *)b.out,
                                                               (TW *)b.w, b.Ls, b.Lw, c, st);
    }
    *launches += 1;
    return cudaGetLastError();
}

template cudaError_t launch_substep_simple<double, double, double>(const StateBufs &,
                                                                   const Coef<double> &,
                                                                   const RKStage &, int, int,
                                                                   cudaStream_t, int *);
template cudaError_t launch_substep_simple<float, float, float>(const StateBufs &,
                                                               const Coef<float> &,
                                                               const RKStage &, int, int,
                                                               cudaStream_t, int *);
template cudaError_t launch_substep_simple<float, float, double>(const StateBufs &,
                                                                const Coef<float> &,
                                                                const RKStage &, int, int,
                                                                cudaStream_t, int *);
template cudaError_t launch_substep_simple<float, float, ffloat>(const StateBufs &,
                                                                const Coef<float> &,
                                                                const RKStage &, int, int,
                                                                cudaStream_t, int *);
template cudaError_t launch_substep_simple<float, double, double>(const StateBufs &,
                                                                 const Coef<float> &,
                                                                 const RKStage &, int, int,
                                                                 cudaStream_t, int *);

template cudaError_t launch_pass2_simple<double, double, double>(const StateBufs &,
                                                              const Coef<double> &, const RKStage &,
                                                              cudaStream_t, int *);
template cudaError_t launch_pass2_simple<float, float, float>(const StateBufs &,
                                                              const Coef<float> &, const RKStage &,
                                                              cudaStream_t, int *);
template cudaError_t launch_pass2_simple<float, float, double>(const StateBufs &,
                                                              const Coef<float> &, const RKStage &,
                                                              cudaStream_t, int *);
template cudaError_t launch_pass2_simple<float, double, double>(const StateBufs &,
                                                              const Coef<float> &, const RKStage &,
                                                              cudaStream_t, int *);

}  // namespace gbfd
