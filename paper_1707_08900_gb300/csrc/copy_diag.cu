// State copies into/out of the padded layout and the FP64 diagnostics
// reductions (mass, kinetic energy, max |u| for the time-step rule, per-field
// rms and max, non-finite flag).
#include <cmath>
#include <cstdint>

#include "kernels.cuh"

namespace gbfd {

namespace {

__device__ __forceinline__ int wrapi(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

// Four consecutive values moved with 16-byte accesses (one float4, or two
// double2), converted on the way.
template <class T>
struct Quad {
    T v[4];
};
template <class T>
__device__ __forceinline__ Quad<T> load_quad(const T *p);
template <>
__device__ __forceinline__ Quad<float> load_quad(const float *p)
{
    const float4 a = *reinterpret_cast<const float4 *>(p);
    return {{a.x, a.y, a.z, a.w}};
}
template <>
__device__ __forceinline__ Quad<double> load_quad(const double *p)
{
    const double2 a = reinterpret_cast<const double2 *>(p)[0];
    const double2 b = reinterpret_cast<const double2 *>(p)[1];
    return {{a.x, a.y, b.x, b.y}};
}
template <class T>
__device__ __forceinline__ void store_quad(T *p, const T (&v)[4]);
template <>
__device__ __forceinline__ void store_quad(float *p, const float (&v)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void store_quad(double *p, const double (&v)[4])
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}

constexpr int COPY_WARPS = 8;  // rows per block: one warp per row

// Every padded row (interior and ghost rows, interior and ghost columns) of
// every field from the compact source; ghosts take the periodic image.  One
// warp per destination row; VEC: source rows 16-byte aligned (nx % 4 == 0
// and an aligned base), so the interior moves in 16-byte accesses.  The
// source may be device memory or pinned host memory mapped into the device
// address space.
template <class TD, class TSrc, bool VEC>
__global__ void __launch_bounds__(32 * COPY_WARPS) k_scatter(const TSrc *__restrict__ src,
                                                            TD *__restrict__ dst, Layout L,
                                                            long long nrows)
{
    const long long row = (long long)blockIdx.x * COPY_WARPS + threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    if (row >= nrows)
        return;
    const int Y = (int)(row % L.rows);
    const long long fz = row / L.rows;
    const int z = (int)(fz % L.nz), f = (int)(fz / L.nz);
    const int y = wrapi(Y - GY, L.ny);
    const TSrc *s = src + (((long long)f * L.nz + z) * L.ny + y) * L.nx;
    TD *d = dst + (long long)f * L.fpitch + (long long)z * L.plane + (long long)Y * L.P;
    if (VEC) {
        for (int x = 4 * lane; x < L.nx; x += 4 * 32) {
            const Quad<TSrc> q = load_quad(s + x);
            const TD v[4] = {(TD)q.v[0], (TD)q.v[1], (TD)q.v[2], (TD)q.v[3]};
            store_quad(d + GX + x, v);
        }
    } else {
        for (int x = lane; x < L.nx; x += 32)
            d[GX + x] = (TD)s[x];
    }
    if (lane < 2 * GX) {
        const int X = lane < GX ? lane : L.nx + lane;
        d[X] = (TD)s[wrapi(X - GX, L.nx)];
    }
}

// Interior rows back to the compact layout; one warp per row.
template <class TS, class TD, bool VEC>
__global__ void __launch_bounds__(32 * COPY_WARPS) k_gather(const TS *__restrict__ src,
                                                           TD *__restrict__ dst, Layout L,
                                                           long long nrows)
{
    const long long row = (long long)blockIdx.x * COPY_WARPS + threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    if (row >= nrows)
        return;
    const int y = (int)(row % L.ny);
    const long long fz = row / L.ny;
    const int z = (int)(fz % L.nz), f = (int)(fz / L.nz);
    const TS *s = src + lidx(L, f, z, y, 0);
    TD *d = dst + row * L.nx;
    if (VEC) {
        for (int x = 4 * lane; x < L.nx; x += 4 * 32) {
            const Quad<TS> q = load_quad(s + x);
            const TD v[4] = {(TD)q.v[0], (TD)q.v[1], (TD)q.v[2], (TD)q.v[3]};
            store_quad(d + x, v);
        }
    } else {
        for (int x = lane; x < L.nx; x += 32)
            d[x] = (TD)s[x];
    }
}

// 16-byte accesses need every row start aligned: the compact side's base
// and row length (nx % 4 == 0 keeps rows of 4- and 8-byte values on 16-byte
// boundaries once the base is), the padded side's interior rows are 128-byte
// aligned by construction.
inline bool quad_ok(const void *compact, int nx)
{
    return ((uintptr_t)compact % 16) == 0 && nx % 4 == 0;
}

template <class TD, class TSrc>
cudaError_t scatter_t(const TSrc *src, TD *dst, const Layout &L, int nf, cudaStream_t stream)
{
    const long long nrows = (long long)nf * L.nz * L.rows;
    const dim3 grid((unsigned)((nrows + COPY_WARPS - 1) / COPY_WARPS)), block(32 * COPY_WARPS);
    if (quad_ok(src, L.nx))
        k_scatter<TD, TSrc, true><<<grid, block, 0, stream>>>(src, dst, L, nrows);
    else
        k_scatter<TD, TSrc, false><<<grid, block, 0, stream>>>(src, dst, L, nrows);
    return cudaGetLastError();
}

template <class TS, class TD>
cudaError_t gather_t(const TS *src, TD *dst, const Layout &L, int nf, cudaStream_t stream)
{
    const long long nrows = (long long)nf * L.nz * L.ny;
    const dim3 grid((unsigned)((nrows + COPY_WARPS - 1) / COPY_WARPS)), block(32 * COPY_WARPS);
    if (quad_ok(dst, L.nx))
        k_gather<TS, TD, true><<<grid, block, 0, stream>>>(src, dst, L, nrows);
    else
        k_gather<TS, TD, false><<<grid, block, 0, stream>>>(src, dst, L, nrows);
    return cudaGetLastError();
}

// ------------------------------------------------------ ghost planes in z

// With walls in z (Layout::gz = GZW): the ghost planes of nf fields as the
// mirror images of the interior about the wall points z = 0 and z = nz - 1,
// f(-k) = p_f f(k) and f(nz - 1 + k) = p_f f(nz - 1 - k), k = 1..3, where
// p_f = -1 for the fields flagged in odd_mask (bit f) and +1 otherwise.  Whole
// padded planes are copied (ghost rows and columns included: the producing
// kernel has already made them periodic copies).  One thread per 16 bytes of
// the 2 GZW ghost planes of every field (a padded plane is a whole number of
// 128-byte rows).
template <class T>
__global__ void __launch_bounds__(256) k_fill_ghosts_z(T *__restrict__ origin, Layout L, int nf,
                                                      int odd_mask)
{
    constexpr int V = 16 / sizeof(T);
    const long long pv = L.plane / V;  // 16-byte vectors per plane
    const long long total = (long long)nf * 2 * GZW * pv;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long e = i % pv;
        long long r = i / pv;
        const int k = 1 + (int)(r % GZW);
        r /= GZW;
        const int side = (int)(r % 2);
        const int f = (int)(r / 2);
        const int zsrc = side ? L.nz - 1 - k : k;
        const int zdst = side ? L.nz - 1 + k : -k;
        const T *src = origin + (long long)f * L.fpitch + (long long)zsrc * L.plane;
        T *dst = origin + (long long)f * L.fpitch + (long long)zdst * L.plane;
        // a plane is the P * rows values from its (Y, X) = (0, 0) element,
        // which is 16-byte aligned (128 - GX w bytes past a 128-byte boundary)
        uint4 v = reinterpret_cast<const uint4 *>(src)[e];
        if ((odd_mask >> f) & 1) {
            T *t = reinterpret_cast<T *>(&v);
#pragma unroll
            for (int j = 0; j < V; ++j)
                t[j] = -t[j];
        }
        reinterpret_cast<uint4 *>(dst)[e] = v;
    }
}

}  // namespace

cudaError_t launch_fill_ghosts_z(void *origin, const Layout &L, int nf, int odd_mask,
                                 cudaStream_t stream, int *launches)
{
    if (!L.gz)
        return cudaSuccess;
    const long long total = (long long)nf * 2 * GZW * (L.plane * L.w / 16);
    const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    if (L.w == 8)
        k_fill_ghosts_z<double><<<blocks, 256, 0, stream>>>((double *)origin, L, nf, odd_mask);
    else
        k_fill_ghosts_z<float><<<blocks, 256, 0, stream>>>((float *)origin, L, nf, odd_mask);
    *launches += 1;
    return cudaGetLastError();
}

namespace {

// ---------------------------------------------------------------- reductions

constexpr int DIAG_THREADS = 256;
constexpr int NQ = 16;  // reduced quantities per block

// q[0] sum rho, q[1] sum rho|u|^2/2, q[2] max|u|^2, q[3] sum |u|^2,
// q[4..8] sum f^2, q[9..13] max |f|, q[14] non-finite count.
template <class TS>
__global__ void __launch_bounds__(DIAG_THREADS) k_diag_partial(const TS *__restrict__ st,
                                                                Layout L, int nf,
                                                                double *__restrict__ part)
{
    double q[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i)
        q[i] = 0.0;
    const long long nrows = (long long)L.nz * L.ny;
    for (long long r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int z = (int)(r / L.ny), y = (int)(r % L.ny);
        for (int x = threadIdx.x; x < L.nx; x += blockDim.x) {
            double v[5];
#pragma unroll
            for (int f = 0; f < 5; ++f)
                v[f] = f < nf ? (double)st[lidx(L, f, z, y, x)] : 0.0;
            const double rho = exp(v[0]);
            const double uu = v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
            q[0] += rho;
            q[1] += 0.5 * rho * uu;
            q[2] = fmax(q[2], uu);
            q[3] += uu;
#pragma unroll
            for (int f = 0; f < 5; ++f) {
                q[4 + f] += v[f] * v[f];
                q[9 + f] = fmax(q[9 + f], fabs(v[f]));
                if (!isfinite(v[f]))
                    q[14] += 1.0;
            }
        }
    }
    // fixed-order block tree reduction
    __shared__ double sh[DIAG_THREADS];
    for (int i = 0; i < 15; ++i) {
        const bool ismax = (i == 2) || (i >= 9 && i <= 13);
        sh[threadIdx.x] = q[i];
        __syncthreads();
        for (int s = DIAG_THREADS / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                const double a = sh[threadIdx.x], b = sh[threadIdx.x + s];
                sh[threadIdx.x] = ismax ? fmax(a, b) : a + b;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0)
            part[(long long)blockIdx.x * NQ + i] = sh[0];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(DIAG_THREADS) k_diag_final(const double *__restrict__ part,
                                                              int nblocks, long long npts,
                                                              double dv, double *__restrict__ out)
{
    __shared__ double sh[DIAG_THREADS];
    __shared__ double res[NQ];
    for (int i = 0; i < 15; ++i) {
        const bool ismax = (i == 2) || (i >= 9 && i <= 13);
        double a = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += DIAG_THREADS) {
            const double v = part[(long long)b * NQ + i];
            a = ismax ? fmax(a, v) : a + v;
        }
        sh[threadIdx.x] = a;
        __syncthreads();
        for (int s = DIAG_THREADS / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                const double x = sh[threadIdx.x], y = sh[threadIdx.x + s];
                sh[threadIdx.x] = ismax ? fmax(x, y) : x + y;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0)
            res[i] = sh[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double n = (double)npts;
        out[0] = dv * res[0];
        out[1] = dv * res[1];
        out[2] = sqrt(res[2]);
        out[3] = sqrt(res[3] / n);
        for (int f = 0; f < 5; ++f) {
            out[4 + f] = sqrt(res[4 + f] / n);
            out[9 + f] = res[9 + f];
        }
        out[14] = res[14] > 0.0 ? 1.0 : 0.0;
        out[15] = 0.0;
    }
}

}  // namespace

cudaError_t launch_scatter(const void *src, int src_fp64, void *dst, const Layout &L, int nf,
                           cudaStream_t stream, int *launches)
{
    *launches += 1;
    if (L.w == 8)
        return src_fp64 ? scatter_t((const double *)src, (double *)dst, L, nf, stream)
                        : scatter_t((const float *)src, (double *)dst, L, nf, stream);
    return src_fp64 ? scatter_t((const double *)src, (float *)dst, L, nf, stream)
                    : scatter_t((const float *)src, (float *)dst, L, nf, stream);
}

cudaError_t launch_gather(const void *src, const Layout &L, void *dst, int dst_fp64, int nf,
                          cudaStream_t stream, int *launches)
{
    *launches += 1;
    if (L.w == 8)
        return dst_fp64 ? gather_t((const double *)src, (double *)dst, L, nf, stream)
                        : gather_t((const double *)src, (float *)dst, L, nf, stream);
    return dst_fp64 ? gather_t((const float *)src, (double *)dst, L, nf, stream)
                    : gather_t((const float *)src, (float *)dst, L, nf, stream);
}

namespace {

__global__ void k_forcing_tables(int kx, int ky, int kz, double cphi, double sphi, int nx, int ny,
                                 int nz, double2 *__restrict__ tab, float2 *__restrict__ tab32)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx + ny + nz)
        return;
    int n, k, idx;
    if (i < nx) {
        n = nx, k = kx, idx = i;
    } else if (i < nx + ny) {
        n = ny, k = ky, idx = i - nx;
    } else {
        n = nz, k = kz, idx = i - nx - ny;
    }
    // exact integer reduction of the phase k idx / n (in turns)
    long long m = ((long long)k * idx) % n;
    m += m < 0 ? n : 0;
    double sn, cs;
    sincospi(2.0 * (double)m / (double)n, &sn, &cs);
    if (i < nx) {
        const double c2 = cs * cphi - sn * sphi, s2 = sn * cphi + cs * sphi;
        cs = c2;
        sn = s2;
    }
    tab[i] = make_double2(cs, sn);
    tab32[i] = make_float2((float)cs, (float)sn);
}

}  // namespace

cudaError_t launch_forcing_tables(int kx, int ky, int kz, double phi, int nx, int ny, int nz,
                                  double2 *tab, float2 *tab32, cudaStream_t stream,
                                  int *launches)
{
    const int n = nx + ny + nz;
    k_forcing_tables<<<(n + 255) / 256, 256, 0, stream>>>(kx, ky, kz, cos(phi), sin(phi), nx, ny,
                                                           nz, tab, tab32);
    *launches += 1;
    return cudaGetLastError();
}

int diag_blocks(const Layout &L)
{
    const long long rows = (long long)L.nz * L.ny;
    return (int)(rows < 1216 ? rows : 1216);  // 8 blocks per SM on 152 SMs
}

cudaError_t launch_diagnostics(const void *state, const Layout &L, int nf, double dv,
                               double *partials, int nblocks, double *out, cudaStream_t stream,
                               int *launches)
{
    if (L.w == 8)
        k_diag_partial<double><<<nblocks, DIAG_THREADS, 0, stream>>>((const double *)state, L, nf,
                                                                     partials);
    else
        k_diag_partial<float><<<nblocks, DIAG_THREADS, 0, stream>>>((const float *)state, L, nf,
                                                                    partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    k_diag_final<<<1, DIAG_THREADS, 0, stream>>>(partials, nblocks,
                                                 (long long)L.nx * L.ny * L.nz, dv, out);
    *launches += 2;
    return cudaGetLastError();
}

}  // namespace gbfd
