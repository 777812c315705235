// gbfd_diagnostics_noalloc: the FP64 diagnostics reduction for callers that
// cannot allocate device memory.
//
// The regular gbfd_diagnostics reads the state held by a context and keeps
// its per-block partial sums in the context's workspace, which the caller
// allocated.  Some callers have neither: code that runs where cudaMalloc is
// off limits (inside a host callback or another stream-ordered section where
// the implicit device synchronisation of cudaMalloc/cudaFree would stall or
// deadlock, or inside a host framework that only allows allocations through
// its own pool and has none to spare), and that only holds a plain state
// array.  This variant takes that state array and an output buffer and keeps
// its partial sums in a fixed, file-scope device array instead.
//
// Limits and sharing rules:
//  * the scratch array holds the partial sums of at most kMaxBlocks = 1216
//    blocks (16 doubles each, 155,648 bytes); every GPU that loads the library
//    holds it until the process exits;
//  * every call on a device uses the same array and it keeps the previous
//    call's contents; each call overwrites the partial rows it reads before
//    reading them, so nothing has to be cleared, but calls whose work
//    overlaps on the GPU (different streams without ordering) race on it;
//  * the device address of the array is looked up once per device, on the
//    first call made while that device is current (again if that device's
//    context was replaced, e.g. after cudaDeviceReset, since the array then
//    lives at a new address); make that first call before any stream
//    capture begins, and where allocation is allowed: with lazy module
//    loading it is also the call that loads this file's device code, and
//    that load may allocate device memory for the module (later calls do
//    not).
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/gbfd.h"

namespace gbfd {
void set_global_error(const char *msg);
}

namespace {

constexpr int kMaxBlocks = 1216;
constexpr int kQ = 16;
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_scratch[kMaxBlocks * kQ];

std::mutex g_mu;
double *g_scratch_addr[kMaxDevices];
unsigned long long g_scratch_ctx[kMaxDevices];  // context ID the address belongs to

// Unique ID of the calling thread's current context (0 when it cannot be
// read); IDs are never reused within a process, unlike context handles.
unsigned long long current_context_id()
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (GetCurrent)p;
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (GetId)p;
        looked_up = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx &&
        get_id(ctx, &id) == CUDA_SUCCESS)
        return id;
    return 0;
}

// Device address of g_scratch on the current device: looked up once per
// device, and again when that device's context has changed.
cudaError_t scratch_address(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= kMaxDevices)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    // the runtime binds the device's primary context on first use; the
    // symbol lookup below does that, so read the context ID after it when
    // nothing is cached yet
    const unsigned long long ctx = g_scratch_addr[dev] ? current_context_id() : 0;
    if (!g_scratch_addr[dev] || ctx != g_scratch_ctx[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess)
            return e;
        g_scratch_addr[dev] = static_cast<double *>(p);
        g_scratch_ctx[dev] = current_context_id();
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// q[0] sum rho, q[1] sum rho |u|^2 / 2, q[2] max |u|^2, q[3] sum |u|^2,
// q[4..8] sum f^2, q[9..13] max |f|, q[14] count of non-finite values.
template <class T>
__global__ void __launch_bounds__(kThreads) k_noalloc_partial(const T *__restrict__ st, int nx,
                                                              int ny, int nz, int nf,
                                                              double *__restrict__ part)
{
    double q[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i)
        q[i] = 0.0;
    const long long npts = (long long)nx * ny * nz;
    const long long nrows = (long long)nz * ny;
    for (long long r = blockIdx.x; r < nrows; r += gridDim.x) {
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const long long c = r * nx + x;
            double v[5];
#pragma unroll
            for (int f = 0; f < 5; ++f)
                v[f] = f < nf ? (double)st[f * npts + c] : 0.0;
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
    __shared__ double sh[kThreads];
    for (int i = 0; i < 15; ++i) {
        const bool ismax = (i == 2) || (i >= 9 && i <= 13);
        sh[threadIdx.x] = q[i];
        __syncthreads();
        for (int s = kThreads / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                const double a = sh[threadIdx.x], b = sh[threadIdx.x + s];
                sh[threadIdx.x] = ismax ? fmax(a, b) : a + b;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0)
            part[(long long)blockIdx.x * kQ + i] = sh[0];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads) k_noalloc_final(const double *__restrict__ part,
                                                            int nblocks, long long npts,
                                                            double dv, double *__restrict__ out)
{
    __shared__ double sh[kThreads];
    __shared__ double res[kQ];
    for (int i = 0; i < 15; ++i) {
        const bool ismax = (i == 2) || (i >= 9 && i <= 13);
        double a = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += kThreads) {
            const double v = part[(long long)b * kQ + i];
            a = ismax ? fmax(a, v) : a + v;
        }
        sh[threadIdx.x] = a;
        __syncthreads();
        for (int s = kThreads / 2; s > 0; s >>= 1) {
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

gbfd_status fail(const char *msg)
{
    gbfd::set_global_error(msg);
    return GBFD_ERR_INVALID_ARG;
}

}  // namespace

extern "C" gbfd_status gbfd_diagnostics_noalloc(const void *state, int state_is_fp64, int nx,
                                                int ny, int nz, int nfields, double lx, double ly,
                                                double lz, void *stream, double *out)
{
    if (!state || !out)
        return fail("diagnostics_noalloc: state and out must be device pointers, not NULL");
    if (nfields != 4 && nfields != 5)
        return fail("diagnostics_noalloc: nfields must be 4 or 5");
    if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz > (1LL << 33))
        return fail("diagnostics_noalloc: grid extents must be >= 1 and nx*ny*nz <= 2^33");
    if (!(lx > 0) || !(ly > 0) || !(lz > 0) || !std::isfinite(lx) || !std::isfinite(ly) ||
        !std::isfinite(lz))
        return fail("diagnostics_noalloc: box lengths must be finite and > 0");
    // one block per grid row up to the scratch's kMaxBlocks rows of partial
    // sums; larger grids need no more scratch, since each block walks the
    // rows in a grid-stride loop
    const long long rows = (long long)nz * ny;
    const int nblocks = (int)(rows < kMaxBlocks ? rows : kMaxBlocks);
    double *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        char buf[200];
        snprintf(buf, sizeof buf, "diagnostics_noalloc: scratch address lookup failed: %s",
                 cudaGetErrorString(e));
        gbfd::set_global_error(buf);
        return GBFD_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (state_is_fp64)
        k_noalloc_partial<double><<<nblocks, kThreads, 0, s>>>((const double *)state, nx, ny, nz,
                                                              nfields, scratch);
    else
        k_noalloc_partial<float><<<nblocks, kThreads, 0, s>>>((const float *)state, nx, ny, nz,
                                                             nfields, scratch);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        const double dv = (lx / nx) * (ly / ny) * (lz / nz);
        k_noalloc_final<<<1, kThreads, 0, s>>>(scratch, nblocks, (long long)nx * ny * nz, dv, out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        char buf[200];
        snprintf(buf, sizeof buf, "diagnostics_noalloc: launch failed: %s", cudaGetErrorString(e));
        gbfd::set_global_error(buf);
        return GBFD_ERR_CUDA;
    }
    return GBFD_OK;
}
