// Device throughput probes: the rate at which this GPU retires independent
// FP64 fused multiply-adds on its CUDA cores (the FP64 path's roofline
// denominator: its kernels are bound by that pipe, not by HBM), and the cost
// of one tcgen05 MMA against N (which fixes the convolutions' MMA shape).
// No counterpart in the paper.
#include <cuda_runtime.h>

#include <cstdio>

#include "../../include/gbfd.h"
#include "tcgen05.cuh"
#include "tiled_impl.cuh"

namespace gbfd {
void set_global_error(const char *msg);
}

namespace {

constexpr int kChains = 8;      // independent FMA chains per thread
constexpr int kThreads = 256;

// kChains independent chains x = x * a + b per thread, `iters` rounds; the
// result is written only if it hits an impossible value, so nothing is
// optimised away and nothing is stored in practice.
__global__ void __launch_bounds__(kThreads) k_dfma(double *out, int iters, double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k)
        x[k] = 1e-3 * (threadIdx.x + k);
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int k = 0; k < kChains; ++k)
                x[k] = fma(x[k], a, b);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k)
        s += x[k];
    if (s == -12345.0)
        out[blockIdx.x] = s;
}

// One CTA per SM; its thread 0 issues `reps` x 8 MMAs of M = 128, K = 16,
// N columns (BF16 operands from shared memory, no swizzle, K-major, with the
// convolutions' A strides and 16-byte shifted A starts; FP32 accumulation
// into TMEM) back to back, then waits for their completion; clock64 cycles
// per MMA into cycles[blockIdx.x].  The operand values do not matter (zeros).
constexpr int kMmaA = 32768, kMmaB = 8192;
constexpr int kMaxSms = 1024;
__device__ double g_mma_cycles[kMaxSms];
__device__ int g_mma_err;

template <int N>
__global__ void __launch_bounds__(128, 1) k_mma_rate(double *cycles, int reps, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem, *sB = smem + kMmaA;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kMmaA + kMmaB);
    uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 1);
    for (int i = threadIdx.x; i < (kMmaA + kMmaB) / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(smem)[i] = make_uint4(0, 0, 0, 0);
    if (threadIdx.x == 0) {
        gbfd::tiled::mbar_init(bar, 1);
        gbfd::tiled::fence_mbar_init();
    }
    if (threadIdx.x < 32)
        gbfd::tc::tmem_alloc(slot, 256);
    gbfd::tc::fence_smem_to_async();
    gbfd::tc::fence_before_sync();
    __syncthreads();
    gbfd::tc::fence_after_sync();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(slot);
    if (threadIdx.x == 0) {
        constexpr uint32_t idesc = gbfd::tc::idesc_bf16_f32(128, N);
        // A: row groups 160 bytes apart, K halves 17,280 bytes apart (the
        // convolution's halo box); B: N x 16 in core-matrix order
        const uint64_t a0 = gbfd::tc::smem_desc(gbfd::tc::smem_u32(sA), 17280, 160);
        const uint64_t b0 = gbfd::tc::smem_desc(gbfd::tc::smem_u32(sB), 128, 256);
        const long long t0 = clock64();
#pragma unroll 1
        for (int r = 0; r < reps; ++r) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                gbfd::tc::mma_bf16(tmem, a0 + (uint64_t)j, b0, idesc, 1u);
        }
        gbfd::tc::commit(bar);
        bool ok = false;
        for (long long spin = 0; spin < (1ll << 28); ++spin) {
            if (gbfd::tiled::mbar_try_wait(bar, 0)) {
                ok = true;
                break;
            }
        }
        if (!ok) {
            atomicExch(err, 1);
            // the MMAs may still run: wait for them again, bounded, before
            // the TMEM is released
            for (long long spin = 0; spin < (1ll << 28); ++spin)
                if (gbfd::tiled::mbar_try_wait(bar, 0))
                    break;
        }
        cycles[blockIdx.x] = (double)(clock64() - t0) / (8.0 * reps);
    }
    gbfd::tc::fence_before_sync();
    __syncthreads();
    gbfd::tc::fence_after_sync();
    if (threadIdx.x < 32)
        gbfd::tc::tmem_dealloc(tmem, 256);
}

template <int N>
cudaError_t launch_mma_rate(int sms, cudaStream_t s, double *d_cycles, int *d_err)
{
    static_assert(N % 16 == 0 && N >= 16 && N <= 256, "M = 128 MMA shapes");
    static_assert((N / 8) * 256 <= kMmaB, "B operand inside its buffer");
    constexpr int smem = kMmaA + kMmaB + 64;
    cudaError_t e = cudaFuncSetAttribute(k_mma_rate<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem);
    if (e != cudaSuccess)
        return e;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch warms up
        k_mma_rate<N><<<sms, 128, smem, s>>>(d_cycles, 128, d_err);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace

extern "C" gbfd_status gbfd_tc_mma_cycles(int n, void *stream, double *cycles)
{
    if (!cycles) {
        gbfd::set_global_error("tc_mma_cycles: cycles is NULL");
        return GBFD_ERR_INVALID_ARG;
    }
    *cycles = 0.0;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms <= 0) {
        gbfd::set_global_error("tc_mma_cycles: device query failed");
        return GBFD_ERR_CUDA;
    }
    if (sms > kMaxSms)
        sms = kMaxSms;
    cudaStream_t s = (cudaStream_t)stream;
    // results in fixed device arrays (no allocation)
    double *d_cycles = nullptr;
    int *d_err = nullptr;
    e = cudaGetSymbolAddress((void **)&d_cycles, g_mma_cycles);
    if (e == cudaSuccess)
        e = cudaGetSymbolAddress((void **)&d_err, g_mma_err);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(d_err, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        switch (n) {
        case 16: e = launch_mma_rate<16>(sms, s, d_cycles, d_err); break;
        case 32: e = launch_mma_rate<32>(sms, s, d_cycles, d_err); break;
        case 48: e = launch_mma_rate<48>(sms, s, d_cycles, d_err); break;
        case 64: e = launch_mma_rate<64>(sms, s, d_cycles, d_err); break;
        case 96: e = launch_mma_rate<96>(sms, s, d_cycles, d_err); break;
        case 128: e = launch_mma_rate<128>(sms, s, d_cycles, d_err); break;
        case 256: e = launch_mma_rate<256>(sms, s, d_cycles, d_err); break;
        default:
            gbfd::set_global_error("tc_mma_cycles: N must be 16, 32, 48, 64, 96, 128 or 256");
            return GBFD_ERR_INVALID_ARG;
        }
    }
    double h[kMaxSms];
    int herr = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, d_cycles, sms * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess || herr) {
        char buf[160];
        snprintf(buf, sizeof buf, "tc_mma_cycles: %s",
                 herr ? "a wait gave up" : cudaGetErrorString(e));
        gbfd::set_global_error(buf);
        return herr ? GBFD_ERR_TIMEOUT : GBFD_ERR_CUDA;
    }
    double sum = 0.0;
    for (int i = 0; i < sms; ++i)
        sum += h[i];
    *cycles = sum / sms;
    return GBFD_OK;
}

extern "C" gbfd_status gbfd_fp64_fma_rate(void *stream, double *tflops)
{
    if (!tflops) {
        gbfd::set_global_error("fp64_fma_rate: tflops is NULL");
        return GBFD_ERR_INVALID_ARG;
    }
    *tflops = 0.0;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms <= 0) {
        gbfd::set_global_error("fp64_fma_rate: device query failed");
        return GBFD_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = sms * 8, iters = 256;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        gbfd::set_global_error("fp64_fma_rate: event creation failed");
        return GBFD_ERR_CUDA;
    }
    float best = 0.f;
    for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, s);
        k_dfma<<<blocks, kThreads, 0, s>>>(nullptr, iters, 0.9999999, 1e-7);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep >= 2 && (best == 0.f || ms < best))
            best = ms;  // the first two launches warm up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || best <= 0.f) {
        char buf[160];
        snprintf(buf, sizeof buf, "fp64_fma_rate: %s", cudaGetErrorString(e));
        gbfd::set_global_error(buf);
        return GBFD_ERR_CUDA;
    }
    const double flops = 2.0 * kChains * 16.0 * iters * (double)blocks * kThreads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return GBFD_OK;
}
